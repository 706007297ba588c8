"""The P1 coarse space on the Kuhn simplices of the box mesh (Remark 2.1) through the C ABI,
against the oracle: host elements and basis values bit for bit (the lowest-element rule and
the barycentric values), coarse dofs, the Galerkin matrix, restriction, coarse solve and
prolongation (the fused kernels form the P1 values from the local coordinates on the fly),
star solves with element patches (the host simplex must have the star's mesh node as a
vertex) and support patches, B, whole solves one at a time and in blocks of right-hand
sides, and the rates of the rate experiment.  Stars sit at every mesh node (Section 4.1):
with P1 element patches and stars at the interior mesh nodes only, a node in a corner box
whose host simplex has only boundary vertices lies in no star."""
import functools
from dataclasses import replace

import numpy as np
import pytest

from oracle.pcg import convergence_rates
from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw
from parity_checks import check_entries, check_star_term, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300 import spnet  # noqa: E402
from paper_2207_07488_gb300.experiments import pcg_rates  # noqa: E402

PREC = {"fp64": spnet.PREC_FP64, "mixed": spnet.PREC_MIXED}


def _grid(patch):
    return replace(nw.grid_heat_problem(5, 0.25, patch=patch), coarse="p1")


def _fibre2d():
    return replace(nw.config1(), coarse="p1", star_set="all")


def _small3d():
    net = nw.fiber_network_3d(1500, 0.2, 0.01, seed=31)
    return replace(nw.scalar_band_problem(net, 0.25, name="small3d"), coarse="p1", star_set="all")


def _small3d_support():
    return replace(_small3d(), patch="support")


def _truss():
    net = nw.fiber_network_3d(1200, 0.25, 0.02, seed=41, keep="clamped_x")
    return replace(nw.truss_band_problem(net, 0.25, name="truss"), coarse="p1", star_set="all")


CASES = {
    "grid_support": lambda: _grid("support"),
    "grid_element": lambda: _grid("element"),
    "fibre2d": _fibre2d,
    "small3d": _small3d,
    "small3d_support": _small3d_support,
    "truss": _truss,
}


@functools.lru_cache(maxsize=None)
def problem(name):
    return CASES[name]()


@functools.lru_cache(maxsize=None)
def oracle(name):
    return OracleSolver(problem(name), local="dense")


def _pc(p, prec, batch_rhs=1):
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=PREC[prec],
                              star_set=spnet.STARS_ALL if p.star_set == "all" else spnet.STARS_INTERIOR,
                              patch=p.patch, coarse=p.coarse, batch_rhs=batch_rhs)
    return op, pc


@functools.lru_cache(maxsize=None)
def lib(name, prec):
    return _pc(problem(name), prec)


@pytest.mark.parametrize("name", list(CASES))
def test_elements_and_p1_values_exact(name):
    o = oracle(name)
    _, pc = lib(name, "fp64")
    cs = o.B.coarse
    assert cs.space == "p1"
    nH = cs.nH
    e = cs.elem
    lin = e[:, 0] + nH[0] * e[:, 1] + (nH[0] * nH[1] * e[:, 2] if e.shape[1] == 3 else 0)
    np.testing.assert_array_equal(pc.export(spnet.EXPORT_ELEMENTS), lin)
    np.testing.assert_array_equal(pc.export(spnet.EXPORT_Q1), cs.W)


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_dofs_and_galerkin(name):
    o = oracle(name)
    _, pc = lib(name, "fp64")
    np.testing.assert_array_equal(pc.export(spnet.EXPORT_COARSE_MAP), o.B.coarse.coarse_index.ravel())
    assert pc.info.m0 == o.B.coarse.m0
    A0 = pc.export(spnet.EXPORT_A0)
    ref = o.B.coarse.A0
    assert np.abs(A0 - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_restrict_coarse_prolong(name, prec):
    o = oracle(name)
    _, pc = lib(name, prec)
    r = np.random.default_rng(2).standard_normal(o.A.shape[0])
    R0 = o.B.coarse.R0
    rc = pc.restrict(r)
    check_entries(rc, R0 @ r, 1e-13 * (abs(R0) @ np.abs(r)) + 1e-300, "restrict")
    zc = pc.coarse(rc)
    ref = o.B.coarse_solve(R0 @ r)
    assert rel(zc, ref) <= (1e-10 if prec == "fp64" else 2e-4)
    z = pc.prolong(ref)
    check_entries(z, R0.T @ ref, 1e-13 * (abs(R0.T) @ np.abs(ref)) + 1e-300, "prolong")


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_star_solves_and_B(name, prec):
    o = oracle(name)
    _, pc = lib(name, prec)
    r = np.random.default_rng(3).standard_normal(o.A.shape[0])
    check_star_term(o, r, pc.stars(r), prec)
    assert rel(pc.apply(r), o.B.apply(r)) <= (1e-10 if prec == "fp64" else 2e-4)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_solve_parity(name, prec):
    p = problem(name)
    o = oracle(name)
    op, pc = lib(name, prec)
    u, st = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-8, maxit=1000)
    ref = o.solve(rtol=1e-8, maxit=1000)
    assert st[0].converged and st[0].relres <= 1e-8
    assert rel(u, ref.u) <= 1e-6
    if prec == "fp64":
        assert abs(st[0].iterations - ref.iters) <= 1


@pytest.mark.parametrize("name", ["fibre2d", "small3d", "truss"])
def test_blocks_of_right_hand_sides(name):
    """The batched update and combine kernels form the P1 values too: four right-hand
    sides stepped together, each against the oracle's solve of it."""
    p = problem(name)
    o = oracle(name)
    op, pc = _pc(p, "mixed", batch_rhs=4)
    rng = np.random.default_rng(7)
    F = rng.uniform(0.0, 1.0, size=(4, p.n_dof))
    U, st = spnet.pcg_solve(op, pc, F, np.tile(p.dirichlet_vals, (4, 1)), rtol=1e-8, maxit=1000)
    for j in range(4):
        ref = o.solve(f=F[j], rtol=1e-9, maxit=1000)
        assert st[j].converged
        assert rel(U[j], ref.u) <= 1e-6
    pc.close()
    op.close()


def test_rates_against_the_oracle():
    p = problem("grid_support")
    o = oracle("grid_support")
    import scipy.sparse.linalg as spla
    b = o.rhs()
    u = spla.spsolve(o.A.tocsc(), b)
    its = []
    o.solve(rtol=1e-13, callback=lambda x, i: its.append(x.copy()))
    taus, errs = convergence_rates(o.A, u, its)
    last = int(np.nonzero(errs <= 1e-8 * errs[0])[0][0])
    got = pcg_rates(p)
    assert got["steps"] == last
    np.testing.assert_allclose(got["taus"], taus[: last - 1], atol=1e-6)


def test_unknown_coarse_space_is_rejected():
    p = problem("grid_support")
    op = spnet.Operator.from_problem(p)
    with pytest.raises(spnet.SpnetError):
        spnet.Preconditioner(op, p.H, p.gamma_faces, coarse=7)
    op.close()


def test_dofs_in_no_star_are_rejected():
    """P1 element patches with stars at the interior mesh nodes only leave the nodes of some
    corner simplices in no star; set-up says so instead of building a singular B."""
    p = replace(nw.config1(), coarse="p1")
    o = OracleSolver(p)
    covered = np.zeros(o.A.shape[0], dtype=bool)
    for S in o.B.stars:
        covered[S] = True
    assert not covered.all()   # the oracle's stars miss some dofs too
    op = spnet.Operator.from_problem(p)
    with pytest.raises(spnet.SpnetError) as e:
        spnet.Preconditioner(op, p.H, p.gamma_faces, star_set=spnet.STARS_INTERIOR, coarse="p1")
    assert e.value.code == spnet.ERR_BAD_INPUT
    op.close()
