"""Parity of every step of the CUDA path with the CPU oracle, through the C ABI.

Each step of the preconditioned iteration is compared on its own (assembly,
the free split and SpMV, host elements and Q1 values, coarse dofs, stars, the
Galerkin matrix, restriction, coarse solve, prolongation, star solves, B),
then whole solves.  Integer and index results must match exactly; FP64
results to a few ulps of the data; FP32 (mixed) local and coarse solves to
the FP32 factorisation error; every solution to a recomputed relative
residual of 1e-8 and a relative error of at most 1e-6 against the oracle.
"""
import functools

import numpy as np
import pytest

from oracle import operator as oop
from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw
from parity_checks import check_entries, check_star_term, rel, star_scale

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300 import spnet  # noqa: E402

PREC = {"fp64": spnet.PREC_FP64, "mixed": spnet.PREC_MIXED}


def _small3d():
    net = nw.fiber_network_3d(1500, 0.2, 0.01, seed=31)
    return nw.scalar_band_problem(net, 0.25, name="small3d")


def _truss():
    net = nw.fiber_network_3d(1200, 0.25, 0.02, seed=41, keep="clamped_x")
    return nw.truss_band_problem(net, 0.25, name="truss")


def _grid():
    return nw.grid_heat_problem(5, 0.25)


def _grid_element():
    return nw.grid_heat_problem(5, 0.25, patch="element")


CASES = {
    "c1": nw.config1,
    "small3d": _small3d,
    "truss": _truss,
    "grid_all": _grid,
    "grid_element": _grid_element,
}


@functools.lru_cache(maxsize=None)
def problem(name):
    return CASES[name]()


@functools.lru_cache(maxsize=None)
def oracle(name):
    return OracleSolver(problem(name), local="dense")


@functools.lru_cache(maxsize=None)
def lib(name, prec):
    p = problem(name)
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=PREC[prec],
                              star_set=spnet.STARS_ALL if p.star_set == "all" else spnet.STARS_INTERIOR,
                              patch=p.patch)
    return op, pc


@pytest.mark.parametrize("name", list(CASES))
def test_assembly_matches_oracle(name):
    p = problem(name)
    net = p.net
    if p.model == "scalar":
        rp, col, val = spnet.assemble(spnet.MODEL_SCALAR, net.n_nodes, net.edges, net.cond)
    else:
        rp, col, val = spnet.assemble(spnet.MODEL_TRUSS3, net.n_nodes, net.edges, net.stiff, net.dirs)
    K = oop.assemble(p).tocsr()
    K.sum_duplicates()
    K.sort_indices()
    # the library keeps explicit zeros of the pattern; compare as dense rows on the union pattern
    assert rp[-1] >= K.nnz
    import scipy.sparse as sp
    Kl = sp.csr_matrix((val, col, rp), shape=K.shape)
    D = (Kl - K).tocoo()
    scale = np.abs(K.data).max()
    assert np.abs(D.data).max(initial=0.0) <= 1e-14 * scale
    # rows sorted strictly ascending, diagonal present
    for i in range(0, K.shape[0], max(1, K.shape[0] // 50)):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c


@pytest.mark.parametrize("name", list(CASES))
def test_free_split_and_spmv(name):
    o = oracle(name)
    op, _ = lib(name, "fp64")
    assert op.info.n_free == o.A.shape[0]
    assert op.info.nnz_ff >= o.A.nnz
    x = np.random.default_rng(1).standard_normal(o.A.shape[0])
    y = op.spmv(x)
    ref = o.A @ x
    bound = (abs(o.A) @ np.abs(x)) * 1e-14
    assert np.all(np.abs(y - ref) <= bound + 1e-300)


@pytest.mark.parametrize("name", list(CASES))
def test_elements_and_q1_values_exact(name):
    o = oracle(name)
    _, pc = lib(name, "fp64")
    cs = o.B.coarse
    nH = cs.nH
    e = cs.elem
    lin = e[:, 0] + nH[0] * e[:, 1] + (nH[0] * nH[1] * e[:, 2] if e.shape[1] == 3 else 0)
    np.testing.assert_array_equal(pc.export(spnet.EXPORT_ELEMENTS), lin)
    np.testing.assert_array_equal(pc.export(spnet.EXPORT_Q1), cs.W)


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_dofs_and_stars_exact(name):
    o = oracle(name)
    _, pc = lib(name, "fp64")
    np.testing.assert_array_equal(pc.export(spnet.EXPORT_COARSE_MAP), o.B.coarse.coarse_index.ravel())
    assert pc.info.m0 == o.B.coarse.m0
    if problem(name).patch == "element":
        np.testing.assert_array_equal(pc.export(spnet.EXPORT_STAR_MESH), np.array(o.B.star_mesh))
        np.testing.assert_array_equal(pc.export(spnet.EXPORT_STAR_SIZES), o.B.star_sizes)
    else:
        # support patches: the library keeps each star's element patch and leaves the dofs
        # off the support out of the solve; its stars are the non-empty element patches
        from oracle.coarse import mesh_multi
        from oracle.schwarz import star_dofs, star_mesh_nodes
        nH = o.B.nH
        mesh, sizes = [], []
        for k in star_mesh_nodes(nH, problem(name).star_set):
            S = star_dofs(o.B.coarse.elem, mesh_multi(k, nH), nH)
            if S.size:
                mesh.append(k)
                sizes.append(S.size)
        np.testing.assert_array_equal(pc.export(spnet.EXPORT_STAR_MESH), np.array(mesh))
        np.testing.assert_array_equal(pc.export(spnet.EXPORT_STAR_SIZES), np.array(sizes))
        assert set(o.B.star_mesh) <= set(mesh) and sum(o.B.star_sizes) < sum(sizes)


@pytest.mark.parametrize("name", list(CASES))
def test_galerkin_matrix(name):
    o = oracle(name)
    _, pc = lib(name, "fp64")
    A0 = pc.export(spnet.EXPORT_A0)
    ref = o.B.coarse.A0
    assert np.abs(A0 - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_restrict_coarse_prolong(name, prec):
    o = oracle(name)
    _, pc = lib(name, prec)
    rng = np.random.default_rng(2)
    r = rng.standard_normal(o.A.shape[0])
    R0 = o.B.coarse.R0
    # restriction and prolongation are FP64 sums of at most a few thousand products:
    # every entry within 1e-13 of the sum of the magnitudes
    rc = pc.restrict(r)
    check_entries(rc, R0 @ r, 1e-13 * (abs(R0) @ np.abs(r)) + 1e-300, "restrict")
    zc = pc.coarse(rc)
    ref = o.B.coarse_solve(rc)
    # A_0^{-1} applied in FP64 or FP32 (cond(A_0) is at most a few hundred here): every
    # entry within the precision's error of the largest entry
    tol = 1e-10 if prec == "fp64" else 2e-4
    check_entries(zc, ref, tol * np.abs(ref).max(), "coarse")
    z = pc.prolong(zc)
    check_entries(z, R0.T @ zc, 1e-13 * (abs(R0).T @ np.abs(zc)) + 1e-300, "prolong")


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_star_solves_and_B(name, prec):
    o = oracle(name)
    _, pc = lib(name, prec)
    r = np.random.default_rng(3).standard_normal(o.A.shape[0])
    sref = check_star_term(o, r, pc.stars(r), prec)
    # B r = coarse term + star term, each entry within the error of both parts
    cref = o.B.coarse_term(r)
    got = pc.apply(r)
    tol = 1e-9 if prec == "fp64" else 2e-4
    if prec == "fp64":
        check_entries(got, cref + sref, 1e-9 * (star_scale(o, r) + np.abs(cref).max()), "B")
    else:
        assert rel(got, cref + sref) <= tol


def _solve_both(name, prec, rtol=1e-8):
    p = problem(name)
    o = oracle(name)
    op, pc = lib(name, prec)
    ref = o.solve(rtol=rtol, flexible=(prec == "mixed"))
    u, st = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=rtol)
    return p, o, ref, u, st[0]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_solve_parity(name, prec):
    p, o, ref, u, st = _solve_both(name, prec)
    assert st.converged == 1 and st.relres <= 1e-8
    # the recomputed residual, checked on the host with the oracle's operator
    x = u[o.free]
    b = o.rhs()
    assert np.linalg.norm(b - o.A @ x) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    assert rel(u, ref.u) <= 1e-6
    np.testing.assert_array_equal(u[p.dirichlet_dofs], p.dirichlet_vals)
    if prec == "fp64":
        assert abs(st.iterations - ref.iters) <= 1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bitwise_reproducible_and_device_arrays(prec):
    name = "small3d"
    p = problem(name)
    op, pc = lib(name, prec)
    u1, _ = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals)
    u2, _ = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals)
    np.testing.assert_array_equal(u1, u2)
    f = torch.from_numpy(p.f).cuda()
    g = torch.from_numpy(p.dirichlet_vals).cuda()
    u3, _ = spnet.pcg_solve(op, pc, f, g)
    np.testing.assert_array_equal(u3.cpu().numpy(), u1)
    # a fresh operator and preconditioner built from device arrays gives the same bits
    op2 = spnet.Operator.from_problem(p, device=True)
    pc2 = spnet.Preconditioner(op2, p.H, p.gamma_faces, precision=PREC[prec])
    u4, _ = spnet.pcg_solve(op2, pc2, f, g)
    np.testing.assert_array_equal(u4.cpu().numpy(), u1)


def test_single_star_converges_in_two_steps():
    net = nw.fiber_network_2d(70, 0.25, seed=5)
    p = nw.scalar_band_problem(net, 0.5)
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_FP64)
    assert pc.info.n_stars == 1
    u, st = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-10)
    assert st[0].iterations <= 2 and st[0].converged


def test_multiple_rhs_and_initial_guess():
    name = "c1"
    p = problem(name)
    op, pc = lib(name, "mixed")
    rng = np.random.default_rng(9)
    F = rng.uniform(0, 1, size=(3, p.n_dof))
    G = np.tile(p.dirichlet_vals, (3, 1))
    U, st = spnet.pcg_solve(op, pc, F, G)
    o = oracle(name)
    for k in range(3):
        ref = o.solve(f=F[k], g=G[k], rtol=1e-8, flexible=True)
        assert rel(U[k], ref.u) <= 1e-6 and st[k].relres <= 1e-8
    # warm start from the solution: converges at once
    U2, st2 = spnet.pcg_solve(op, pc, F, G, x0=U)
    assert all(s.iterations <= 1 for s in st2)


def test_errors_are_reported():
    p = problem("c1")
    op, _ = lib("c1", "fp64")
    with pytest.raises(spnet.SpnetError) as ei:
        spnet.Preconditioner(op, 0.3, p.gamma_faces)
    assert ei.value.code == -8
    net = p.net
    rp, col, val = spnet.assemble(spnet.MODEL_SCALAR, net.n_nodes, net.edges, net.cond)
    free = np.setdiff1d(np.arange(net.n_nodes), p.dirichlet_dofs)
    row = int(free[10])
    ks = [k for k in range(rp[row], rp[row + 1]) if col[k] != row and col[k] in set(free.tolist())]
    # an asymmetric K_II is rejected
    val2 = val.copy()
    val2[ks[0]] += 0.25
    with pytest.raises(spnet.SpnetError) as ei:
        spnet.Operator(2, 1, net.coords, rp, col, val2, p.dirichlet_dofs, net.domain)
    assert ei.value.code == -1
    # a non-positive diagonal cannot belong to an SPD K_II
    val3 = val.copy()
    kd = [k for k in range(rp[row], rp[row + 1]) if col[k] == row][0]
    val3[kd] = -1.0
    with pytest.raises(spnet.SpnetError) as ei:
        spnet.Operator(2, 1, net.coords, rp, col, val3, p.dirichlet_dofs, net.domain)
    assert ei.value.code == -2
    # coordinates outside Omega and unsorted Dirichlet lists are bad input
    X = net.coords.copy()
    X[3, 0] = 1.5
    with pytest.raises(spnet.SpnetError) as ei:
        spnet.Operator(2, 1, X, rp, col, val, p.dirichlet_dofs, net.domain)
    assert ei.value.code == -1
    with pytest.raises(spnet.SpnetError) as ei:
        spnet.Operator(2, 1, net.coords, rp, col, val, p.dirichlet_dofs[::-1].copy(), net.domain)
    assert ei.value.code == -1


def test_star_solve_mapping_changes_no_result():
    # each warp solves whole stars, so the warps per block of the star solve (fixed, or
    # picked by timing per size class) changes timing only: the solutions are bitwise equal
    p = problem("small3d")
    sols, wpbs = [], []
    for star_map in (0, 1, 2, 4, 8):
        op = spnet.Operator.from_problem(p)
        pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED, star_map=star_map)
        wpbs.append(pc.info.star_warps_per_block)
        u, st = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals)
        assert st[0].converged
        sols.append(u)
    assert 1 <= wpbs[0] <= 8 and wpbs[1] == 1 and wpbs[2] == 2
    for u in sols[1:]:
        np.testing.assert_array_equal(u, sols[0])
    with pytest.raises(spnet.SpnetError):
        spnet.Preconditioner(spnet.Operator.from_problem(p), p.H, p.gamma_faces, star_map=9)


def test_dependent_coarse_functions():
    # a sparse 3D draw whose truncated coarse functions are linearly dependent (three of
    # them lie in the span of earlier ones): A_0 is singular, P_0 the projection onto the
    # span (Section 4.1).  The library drops the same three in FP64, its P_0 reproduces
    # V_H, its coarse term matches the oracle's entry by entry, and both precisions solve.
    net = nw.fiber_network_3d(1500, 0.2, 0.01, seed=3)
    p = nw.scalar_band_problem(net, 0.25, name="small3d-dependent")
    o = OracleSolver(p, local="dense")
    n_dep = o.B.coarse.m0 - o.B.coarse_kept.size
    assert n_dep == 3
    R0 = o.B.coarse.R0
    rng = np.random.default_rng(8)
    for prec in ("fp64", "mixed"):
        op = spnet.Operator.from_problem(p)
        pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=PREC[prec])
        if prec == "fp64":
            assert pc.info.coarse_dropped == n_dep
            v = R0.T @ rng.standard_normal(R0.shape[0])
            Pv = pc.prolong(pc.coarse(pc.restrict(o.A @ v)))
            assert np.abs(Pv - v).max() <= 1e-9 * np.abs(v).max()
            r = rng.standard_normal(o.A.shape[0])
            ref = o.B.coarse_term(r)
            got = pc.prolong(pc.coarse(pc.restrict(r)))
            check_entries(got, ref, 1e-9 * np.abs(ref).max(), "coarse term")
        else:
            assert pc.info.coarse_dropped >= n_dep
        u, st = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-8)
        assert st[0].converged and st[0].relres <= 1e-8
        ref = o.solve(rtol=1e-8, flexible=(prec == "mixed"))
        assert rel(u, ref.u) <= 1e-6


def test_structural_workload_as_written():
    # the 20000-fibre structural network spans nothing: the clamped component is kept, f = 0
    # and its Dirichlet data are zero, so u = 0; its coarse functions are dependent
    p = nw.config3()
    op = spnet.Operator.from_problem(p)
    for prec in (spnet.PREC_FP64, spnet.PREC_MIXED):
        pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=prec)
        assert pc.info.coarse_dropped > 0
        u, st = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-8)
        assert st[0].converged and np.all(u == 0.0)
        # a load on the free dofs is solved too
        f = np.random.default_rng(1).uniform(0.0, 1.0, p.n_dof)
        u, st = spnet.pcg_solve(op, pc, f, p.dirichlet_vals, rtol=1e-8)
        assert st[0].converged and st[0].relres <= 1e-8
