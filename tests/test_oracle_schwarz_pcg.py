"""Pins of the oracle's Schwarz preconditioner and PCG (no GPU)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from conftest import read_golden
from oracle import operator as op
from oracle.pcg import convergence_rates, k_norm, lanczos_extremes, pcg
from oracle.schwarz import SchwarzPreconditioner
from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw


def _small(seed=5, H=0.25, star_set="interior"):
    net = nw.fiber_network_2d(70, 0.25, seed=seed)
    return nw.scalar_band_problem(net, H, star_set=star_set)


def test_local_and_coarse_terms_are_projections():
    # eq. defPj: P_j v = v for v in V_j; P_0 v = v for v in V_H
    p = _small()
    free, A, _ = op.split(p)
    B = SchwarzPreconditioner(p, free, A)
    rng = np.random.default_rng(0)
    for j, S in enumerate(B.stars):
        v = np.zeros(A.shape[0])
        v[S] = rng.standard_normal(S.size)
        w = np.zeros_like(v)
        w[S] = B.local_solve(j, (A @ v)[S])
        np.testing.assert_allclose(w, v, atol=1e-9 * np.abs(v).max())
    c = rng.standard_normal(B.coarse.m0)
    v = B.coarse.prolong(c)
    np.testing.assert_allclose(B.coarse_term(A @ v), v, atol=1e-9 * np.abs(v).max())


def test_dense_B_symmetric_pd_and_K_symmetric():
    for star_set in ("interior", "all"):
        p = _small(star_set=star_set)
        free, A, _ = op.split(p)
        B = SchwarzPreconditioner(p, free, A)
        Bd = B.dense_B()
        Ad = A.toarray()
        assert np.abs(Bd - Bd.T).max() <= 1e-11 * np.abs(Bd).max()
        assert np.linalg.eigvalsh(0.5 * (Bd + Bd.T))[0] > 0
        # eq. TTsym: P = B A is symmetric in the K inner product, i.e. A B A is symmetric
        ABA = Ad @ Bd @ Ad
        assert np.abs(ABA - ABA.T).max() <= 1e-10 * np.abs(ABA).max()


def test_stars_cover_free_dofs():
    p = nw.config1()
    free, A, _ = op.split(p)
    B = SchwarzPreconditioner(p, free, A)
    assert B.n_stars == 49
    cover = np.zeros(A.shape[0], int)
    for S in B.stars:
        cover[S] += 1
    assert cover.min() >= 1 and cover.max() <= 4


def test_single_star_two_iterations():
    # H = l/2 with interior stars: one star holds every free dof, so B = A^{-1} + R0^T A0^{-1} R0
    # and B A = I + P_0 has eigenvalues {1, 2}: PCG ends in at most two steps.
    p = _small(H=0.5)
    S = OracleSolver(p)
    assert S.B.n_stars == 1 and S.B.stars[0].size == S.A.shape[0]
    res = S.solve(rtol=1e-10)
    assert res.iters <= 2
    ev = np.linalg.eigvals(S.B.dense_B() @ S.A.toarray()).real
    assert np.all(np.min(np.abs(ev[:, None] - np.array([1.0, 2.0])[None]), axis=1) < 1e-8)


def test_pcg_matches_direct_solve():
    p = nw.config1()
    S = OracleSolver(p)
    res = S.solve(rtol=1e-12)
    x = spla.spsolve(S.A.tocsc(), res.b)
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)
    assert res.true_relres <= 1e-12


def test_k_norm_error_monotone_and_chebyshev_bound():
    p = nw.config1()
    S = OracleSolver(p)
    b = S.rhs()
    u = spla.spsolve(S.A.tocsc(), b)
    its = []
    res = S.solve(rtol=1e-10, callback=lambda x, i: its.append(x.copy()))
    taus, errs = convergence_rates(S.A, u, its)
    # Krylov minimisation in the K-norm (Section 4.2): the error never grows
    assert np.all(errs[1:] <= errs[:-1] * (1 + 1e-9))
    # eq. (optimal): |e_l|_K <= 2 ((sqrt(k) - 1)/(sqrt(k) + 1))^l |e_0|_K with kappa the
    # condition number of P = B A, estimated by the Ritz values of the CG-Lanczos matrix
    lmin, lmax = lanczos_extremes(res.alphas, res.betas)
    kappa = lmax / lmin
    q = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    ell = np.arange(errs.size)
    assert np.all(errs <= 2 * q ** ell * errs[0] * (1 + 1e-6))
    # P contains the star projections and P_0: its spectrum reaches 1 or more
    assert lmax >= 1.0 - 1e-6


def test_flexible_equals_standard_for_exact_B():
    p = nw.config1()
    S = OracleSolver(p)
    r1 = S.solve(rtol=1e-10)
    r2 = S.solve(rtol=1e-10, flexible=True)
    assert abs(r1.iters - r2.iters) <= 1
    assert np.linalg.norm(r1.x - r2.x) <= 1e-8 * np.linalg.norm(r1.x)


def test_refinement_invariance_exact_and_bounded_iterations():
    # splitting each edge into k pieces of conductance k*c leaves the solution at the
    # original nodes unchanged (series conductances); Theorem 4.3 has no N in kappa,
    # so the iteration count stays bounded at fixed H.
    base = nw.config1()
    S0 = OracleSolver(base)
    r0 = S0.solve(rtol=1e-10)
    n0 = base.net.n_nodes
    for k in (2, 4):
        net = nw.subdivide(base.net, k)
        p = nw.Problem(net, 1, "scalar", base.dirichlet_dofs, base.dirichlet_vals,
                       np.zeros(net.n_nodes), base.H, base.gamma_faces, base.star_set)
        S = OracleSolver(p)
        r = S.solve(rtol=1e-10)
        np.testing.assert_allclose(r.u[:n0], r0.u, atol=1e-7)
        assert r.iters <= 1.5 * r0.iters + 2


def _grid_rates(k, Hinv):
    p = nw.grid_heat_problem(k, 1.0 / Hinv)
    S = OracleSolver(p, local="sparse")
    b = S.rhs()
    u = spla.spsolve(S.A.tocsc(), b)
    its = []
    S.solve(rtol=1e-12, callback=lambda x, i: its.append(x.copy()))
    taus, errs = convergence_rates(S.A, u, its)
    last = int(np.nonzero(errs < 1e-8 * errs[0])[0][0])
    return taus[: max(1, last - 1)]


def test_paper_grid_rates():
    """Section 6.2, Table lap_conv (grid row), on the paper's own (2^9+1)^2 grid.

    Stars at every mesh node holding the nodes where the node's basis function is
    nonzero; tau_l = |e_l|_K / |e_{l-1}|_K averaged over l >= 2 until the K-norm error
    has fallen by 1e-8.  Mean and worst rate must lie within 0.05 of the table.
    """
    g = read_golden("lap_conv_grid.txt")["rates"]
    for Hinv, tbar, tmax in g:
        t = _grid_rates(9, int(Hinv))
        assert abs(t.mean() - tbar) <= 0.05, (Hinv, t.mean(), tbar)
        assert abs(t.max() - tmax) <= 0.05, (Hinv, t.max(), tmax)


def test_star_membership_hand_worked():
    """Star sets on a 2 x 2-element mesh with nodes on mesh lines and faces (Section 2.3,
    Section 4.1), worked by hand: the half-open host elements, the "element" stars and
    the "support" stars of every mesh node."""
    from oracle.coarse import host_elements, q1_values
    from oracle.schwarz import star_dofs
    g = read_golden("star_membership.txt")
    X, nH, dom = g["nodes"], (2, 2), (1.0, 1.0)
    e = host_elements(X, dom, nH)
    np.testing.assert_array_equal(e, g["hosts"].astype(np.int64))
    W = q1_values(X, dom, nH, e)
    for rule, Wr in (("element", None), ("support", W)):
        for row in g[rule]:
            km = (int(row[0]), int(row[1]))
            want = np.nonzero(row[2:])[0]
            np.testing.assert_array_equal(star_dofs(e, km, nH, Wr), want, err_msg=f"{rule} {km}")
    # the fixture tells both rules apart from closed patches
    assert not np.array_equal(g["closed"], g["element"])
    assert not np.array_equal(g["closed"], g["support"])


@pytest.mark.slow
def test_grid_iterations_bounded_under_refinement():
    # grid 2^6 -> 2^8 at fixed H = 1/8: iteration counts stay within a small band
    counts = []
    for k in (6, 8):
        p = nw.grid_heat_problem(k, 1.0 / 8)
        counts.append(OracleSolver(p, local="sparse").solve(rtol=1e-8).iters)
    assert counts[1] <= 1.5 * counts[0] + 2


def _small_truss():
    net = nw.fiber_network_3d(250, 0.3, 0.03, seed=13, keep="clamped_x")
    return nw.truss_band_problem(net, 0.5)


def test_truss_projection_symmetry_and_direct_solve():
    p = _small_truss()
    S = OracleSolver(p)
    A = S.A
    B = S.B
    rng = np.random.default_rng(2)
    for j, St in enumerate(B.stars):
        v = np.zeros(A.shape[0])
        v[St] = rng.standard_normal(St.size)
        w = np.zeros_like(v)
        w[St] = B.local_solve(j, (A @ v)[St])
        np.testing.assert_allclose(w, v, atol=1e-8 * np.abs(v).max())
    c = rng.standard_normal(B.coarse.m0)
    v = B.coarse.prolong(c)
    np.testing.assert_allclose(B.coarse_term(A @ v), v, atol=1e-8 * np.abs(v).max())
    res = S.solve(rtol=1e-12)
    x = spla.spsolve(A.tocsc(), res.b)
    assert np.linalg.norm(res.x - x) <= 1e-9 * np.linalg.norm(x)
    # the x-displacement data of the upper band are reproduced
    hi = p.net.coords[:, 0] > 0.99
    np.testing.assert_allclose(res.u[3 * np.nonzero(hi)[0]], 0.01)
