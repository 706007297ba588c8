"""Several right-hand sides stepped together (batch_rhs) against the oracle.

The batched path applies the same preconditioner (Sections 4.1-4.2) to k
residuals at once and runs PCG (Section 4.2) on each right-hand side with its
own scalars and stop test.  Checked here:
- z_j = B r_j, the coarse term and the star term, per column, against the
  oracle at the tolerance of the one-vector path (FP64: 1e-10; mixed: the FP32
  factorisation error, 2e-4);
- whole solves per column against the oracle (recomputed residual <= 1e-8,
  relative error <= 1e-6) and the iteration count in FP64;
- a column's result does not depend on the other columns of its block: the
  kernels give each column its own sums in an order fixed by the padded block
  width, so the same column gives the same bits in any block of that width;
- ragged blocks, the largest block (32), a zero right-hand side, a converged
  initial guess, maxit reached, bad options;
- the full-size workload (40000 fibres, H = 1/16, mixed precision): B per
  column against the oracle and the recomputed residual of every column
  checked on the host with the oracle's operator.
"""
import functools

import numpy as np
import pytest

from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300 import spnet  # noqa: E402

PREC = {"fp64": spnet.PREC_FP64, "mixed": spnet.PREC_MIXED}
TOL = {"fp64": 1e-10, "mixed": 2e-4}


def _small3d():
    net = nw.fiber_network_3d(1500, 0.2, 0.01, seed=31)
    return nw.scalar_band_problem(net, 0.25, name="small3d")


def _truss():
    net = nw.fiber_network_3d(1200, 0.25, 0.02, seed=41, keep="clamped_x")
    return nw.truss_band_problem(net, 0.25, name="truss")


CASES = {"c1": nw.config1, "small3d": _small3d, "truss": _truss,
         "grid_all": lambda: nw.grid_heat_problem(5, 0.25)}  # support patches


@functools.lru_cache(maxsize=None)
def problem(name):
    return CASES[name]() if name in CASES else nw.config2()


@functools.lru_cache(maxsize=None)
def oracle(name):
    return OracleSolver(problem(name), local="dense")


@functools.lru_cache(maxsize=None)
def lib(name, prec, batch):
    p = problem(name)
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=PREC[prec], batch_rhs=batch,
                              star_set=spnet.STARS_ALL if p.star_set == "all" else spnet.STARS_INTERIOR,
                              patch=p.patch)
    return op, pc


from parity_checks import check_star_term, rel  # noqa: E402


def _rhs(p, k, seed):
    rng = np.random.default_rng(seed)
    F = rng.uniform(0.0, 1.0, size=(k, p.n_dof))
    G = np.tile(p.dirichlet_vals, (k, 1)) * rng.uniform(0.5, 1.5, size=(k, 1))
    return F, G


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("k", [1, 3, 32])
def test_apply_batch_per_column(name, prec, k):
    o = oracle(name)
    _, pc = lib(name, prec, 1)
    R = np.random.default_rng(10 + k).standard_normal((k, o.A.shape[0]))
    Z = pc.apply_batch(R)
    Zc = pc.apply_batch(R, which=1)
    Zs = pc.apply_batch(R, which=2)
    for j in range(k):
        assert rel(Z[j], o.B.apply(R[j])) <= TOL[prec], j
        assert rel(Zc[j], o.B.coarse_term(R[j])) <= TOL[prec], j
        if j in (0, k - 1):  # element-wise, per star
            check_star_term(o, R[j], Zs[j], prec)
        else:
            assert rel(Zs[j], o.B.star_term(R[j])) <= TOL[prec], j
    # the one-vector path on the same residual: the same preconditioner up to rounding
    assert rel(Z[0], pc.apply(R[0])) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_solve_parity(name, prec):
    p = problem(name)
    o = oracle(name)
    op, pc = lib(name, prec, 4)
    F, G = _rhs(p, 4, 21)
    U, st = spnet.pcg_solve(op, pc, F, G, rtol=1e-8)
    # the oracle's solve of the truss takes half a minute: one column there, every column elsewhere
    against_oracle = (0,) if name == "truss" else range(4)
    for j in range(4):
        assert st[j].converged == 1 and st[j].relres <= 1e-8, j
        b = o.rhs(F[j], G[j])
        assert np.linalg.norm(b - o.A @ U[j][o.free]) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6), j
        np.testing.assert_array_equal(U[j][p.dirichlet_dofs], G[j])
        if j not in against_oracle:
            continue
        ref = o.solve(f=F[j], g=G[j], rtol=1e-8, flexible=(prec == "mixed"))
        assert rel(U[j], ref.u) <= 1e-6, j
        if prec == "fp64":
            assert abs(st[j].iterations - ref.iters) <= 1, (j, st[j].iterations, ref.iters)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_matches_one_at_a_time(prec):
    name = "small3d"
    p = problem(name)
    F, G = _rhs(p, 5, 22)
    op1, pc1 = lib(name, prec, 1)
    U1, st1 = spnet.pcg_solve(op1, pc1, F, G)
    op5, pc5 = lib(name, prec, 5)
    U5, st5 = spnet.pcg_solve(op5, pc5, F, G)
    for j in range(5):
        assert rel(U5[j], U1[j]) <= 1e-7, j
        assert abs(st5[j].iterations - st1[j].iterations) <= 2, j
        assert st5[j].relres <= 1e-8


def test_a_column_does_not_depend_on_its_neighbours():
    name = "small3d"
    p = problem(name)
    F, G = _rhs(p, 9, 23)
    op, pc = lib(name, "mixed", 4)
    Ua, _ = spnet.pcg_solve(op, pc, F[[0, 1, 2, 3]], G[[0, 1, 2, 3]])
    Ub, _ = spnet.pcg_solve(op, pc, F[[4, 0, 5, 6]], G[[4, 0, 5, 6]])
    Uc, _ = spnet.pcg_solve(op, pc, F[[7, 8, 0]], G[[7, 8, 0]])  # 3 columns: the same padded width 4
    np.testing.assert_array_equal(Ua[0], Ub[1])
    np.testing.assert_array_equal(Ua[0], Uc[2])
    Ud, _ = spnet.pcg_solve(op, pc, F[[0, 1, 2, 3]], G[[0, 1, 2, 3]])
    np.testing.assert_array_equal(Ua, Ud)


def test_ragged_blocks_zero_rhs_and_converged_start():
    name = "c1"
    p = problem(name)
    o = oracle(name)
    F, G = _rhs(p, 7, 24)
    F[3] = 0.0
    G[3] = 0.0
    op, pc = lib(name, "mixed", 5)  # blocks of 5 and 2
    U, st = spnet.pcg_solve(op, pc, F, G)
    assert np.all(U[3] == 0.0) and st[3].iterations == 0 and st[3].converged == 1
    for j in range(7):
        assert st[j].converged == 1, j
        if j != 3:
            assert rel(U[j], o.solve(f=F[j], g=G[j], flexible=True).u) <= 1e-6, j
    # from the solutions: every column is converged at the start
    U2, st2 = spnet.pcg_solve(op, pc, F, G, x0=U)
    assert all(s.iterations <= 1 for s in st2)
    np.testing.assert_array_equal(U2[3], U[3])


def test_largest_block_and_remainder():
    name = "c1"
    p = problem(name)
    F, G = _rhs(p, 33, 25)
    op, pc = lib(name, "mixed", 32)  # a block of 32, then one alone
    U, st = spnet.pcg_solve(op, pc, F, G)
    op1, pc1 = lib(name, "mixed", 1)
    U1, _ = spnet.pcg_solve(op1, pc1, F[32:], G[32:])
    np.testing.assert_array_equal(U[32], U1[0])
    assert all(s.converged == 1 and s.relres <= 1e-8 for s in st)


def test_maxit_reached_is_reported():
    name = "small3d"
    p = problem(name)
    F, G = _rhs(p, 3, 26)
    op, pc = lib(name, "fp64", 4)
    U, st = spnet.pcg_solve(op, pc, F, G, maxit=2, raise_on_noconv=False)
    assert all(s.converged == 0 and s.iterations == 2 for s in st)
    with pytest.raises(spnet.SpnetError):
        spnet.pcg_solve(op, pc, F, G, maxit=2)


def test_bad_batch_options():
    p = problem("c1")
    op = spnet.Operator.from_problem(p)
    with pytest.raises(spnet.SpnetError):
        spnet.Preconditioner(op, p.H, p.gamma_faces, batch_rhs=33)
    _, pc = lib("c1", "mixed", 1)
    with pytest.raises(spnet.SpnetError):
        pc.apply_batch(np.zeros((33, op.info.n_free)))


def test_full_size_batched():
    name = "config2"
    p = problem(name)
    o = oracle(name)
    op, pc = lib(name, "mixed", 4)
    R = np.random.default_rng(27).standard_normal((4, o.A.shape[0]))
    Z = pc.apply_batch(R)
    for j in range(4):
        assert rel(Z[j], o.B.apply(R[j])) <= TOL["mixed"], j
    F, G = _rhs(p, 4, 28)
    U, st = spnet.pcg_solve(op, pc, F, G)
    for j in range(4):
        assert st[j].converged == 1 and st[j].relres <= 1e-8, j
        b = o.rhs(F[j], G[j])
        assert np.linalg.norm(b - o.A @ U[j][o.free]) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6), j
