"""Pins of the oracle's mesh, Q1 values, coarse dofs and Galerkin matrix (no GPU)."""
import numpy as np

from conftest import read_golden
from oracle import coarse as co
from oracle import operator as op
from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw


def test_half_open_host_element_cases():
    for l, n, x, want in read_golden("host_element_cases.txt")["cases"]:
        e = co.host_elements(np.array([[x]]), (l,), (int(n),))
        assert int(e[0, 0]) == int(want), (l, n, x)


def test_q1_partition_of_unity_and_linear_reproduction():
    rng = np.random.default_rng(3)
    for d, nH in ((2, (8, 8)), (3, (4, 5, 3))):
        dom = tuple([1.0] * d)
        X = rng.uniform(0, 1, size=(2000, d))
        X[:50] = np.round(X[:50] * np.array(nH)) / np.array(nH)   # nodes on mesh lines
        e = co.host_elements(X, dom, nH)
        W = co.q1_values(X, dom, nH, e)
        assert W.min() >= -1e-15 and W.max() <= 1 + 1e-15
        np.testing.assert_allclose(W.sum(axis=1), 1.0, atol=1e-14)
        # sum_k phi_k(x) y_k = x  (Q1 reproduces affine functions)
        rec = np.zeros_like(X)
        for ci, c in enumerate(co.corner_list(d)):
            y = (e + np.array(c)) / np.array(nH)
            rec += W[:, ci:ci + 1] * y
        np.testing.assert_allclose(rec, X, atol=1e-14)


def _chain_problem(M, Hinv):
    """Chain of M+1 nodes on y = 0 of the unit square, spacing 1/M, no Dirichlet data."""
    h = 1.0 / M
    X = np.stack([np.arange(M + 1) * h, np.zeros(M + 1)], axis=1)
    E = np.stack([np.arange(M), np.arange(1, M + 1)], axis=1).astype(np.int64)
    net = nw.Network(2, X, E, np.zeros(M, np.int8), np.full(M, 1.0 / h), np.full(M, 1.0 / h),
                     np.tile([1.0, 0.0], (M, 1)), (1.0, 1.0))
    return nw.Problem(net, 1, "scalar", np.zeros(0, np.int64), np.zeros(0), np.zeros(M + 1),
                      1.0 / Hinv, (0,))


def test_galerkin_chain_is_1d_fe_stiffness():
    # The Q1 functions restricted to the chain are 1D hat functions; their network
    # energy is exact for piecewise linears, so A_0 is the 1D P1 stiffness matrix.
    Hinv = 4
    p = _chain_problem(64, Hinv)
    free, A, _ = op.split(p)
    cs = co.CoarseSpace(p, free, A)
    assert cs.m0 == Hinv + 1       # mesh nodes on y = H carry no coarse dof
    T = (2 * np.eye(Hinv + 1) - np.eye(Hinv + 1, k=1) - np.eye(Hinv + 1, k=-1)) * Hinv
    T[0, 0] = T[-1, -1] = Hinv
    np.testing.assert_allclose(cs.A0, T, rtol=1e-12, atol=1e-9)


def test_galerkin_neumann_constants_in_kernel():
    net = nw.fiber_network_2d(400, 0.1, seed=21)
    p = nw.Problem(net, 1, "scalar", np.zeros(0, np.int64), np.zeros(0), np.zeros(net.n_nodes),
                   0.25, (0,))
    free, A, _ = op.split(p)
    cs = co.CoarseSpace(p, free, A)
    assert np.abs(cs.A0 @ np.ones(cs.m0)).max() <= 1e-10 * np.abs(cs.A0).max()
    np.testing.assert_allclose(cs.R0.T @ np.ones(cs.m0), 1.0, atol=1e-13)


def test_coarse_dof_count_and_faces():
    p = nw.config1()
    free, A, _ = op.split(p)
    cs = co.CoarseSpace(p, free, A)
    # H = 1/8: mesh nodes off the faces x = 0 and x = 1: 7 x 9
    assert cs.m0 == 7 * 9
    np.testing.assert_allclose(cs.A0, cs.A0.T, atol=1e-12 * np.abs(cs.A0).max())
    np.linalg.cholesky(cs.A0)


def _line_network():
    """Eleven nodes on the line y = 1/4 of the unit square, x = 0, 0.1, .., 1, joined in a
    chain, u = 0 at both ends; H = 1/2.  The coarse dofs sit at mesh nodes (1, j)
    (x = 0 and x = 1 are Dirichlet faces); phi_(1,2) vanishes on the line and is
    dropped, and on the line phi_(1,1) = phi_(1,0) / 3: the two remaining functions
    are linearly dependent and A_0 is singular."""
    x = np.linspace(0.0, 1.0, 11)
    X = np.stack([x, np.full(11, 0.25)], axis=1)
    E = np.stack([np.arange(10), np.arange(1, 11)], axis=1).astype(np.int64)
    net = nw.Network(2, X, E, np.zeros(10, np.int8), np.full(10, 10.0), np.full(10, 10.0),
                     np.tile([1.0, 0.0], (10, 1)), (1.0, 1.0))
    f = np.ones(11)
    return nw.Problem(net, 1, "scalar", np.array([0, 10]), np.zeros(2), f, 0.5,
                      (nw.face_bit(0, 0) | nw.face_bit(0, 1),), "interior")


def _pinv_coarse_term(B, r):
    """R_0^T A_0^+ R_0 r with numpy's pseudo-inverse: the K-orthogonal projection onto
    the span of the truncated basis functions, whatever their dependence."""
    A0p = np.linalg.pinv(B.coarse.A0, rcond=1e-10, hermitian=True)
    return B.coarse.R0.T @ (A0p @ (B.coarse.R0 @ r))


def test_dependent_coarse_functions_are_dropped():
    # Section 4.1: P_0 is the projection onto V_H, a span; dropping the functions that
    # lie in the span of the ones kept before them leaves P_0 unchanged
    from oracle.schwarz import SchwarzPreconditioner
    p = _line_network()
    free, A, _ = op.split(p)
    B = SchwarzPreconditioner(p, free, A)
    assert B.coarse.m0 == 2
    assert np.linalg.matrix_rank(B.coarse.A0) == 1
    np.testing.assert_array_equal(B.coarse_kept, [0])
    rng = np.random.default_rng(3)
    for _ in range(3):
        r = rng.standard_normal(free.size)
        np.testing.assert_allclose(B.coarse_term(r), _pinv_coarse_term(B, r), rtol=1e-12, atol=1e-14)
    # P_0 v = v on V_H (both functions, the dropped one included) and P_0 P_0 = P_0
    Ad = A.toarray()
    for c in (np.array([1.0, 0.0]), np.array([0.0, 1.0]), rng.standard_normal(2)):
        v = B.coarse.prolong(c)
        np.testing.assert_allclose(B.coarse_term(Ad @ v), v, atol=1e-12 * np.abs(v).max())
    w = B.coarse_term(Ad @ rng.standard_normal(free.size))
    np.testing.assert_allclose(B.coarse_term(Ad @ w), w, atol=1e-12 * np.abs(w).max())
    # the whole solve still matches the direct solve
    S = OracleSolver(p)
    res = S.solve(rtol=1e-12)
    np.testing.assert_allclose(res.x, np.linalg.solve(Ad, res.b), rtol=1e-10)


def test_dependent_functions_on_a_sparse_fiber_network():
    # a sparse 3D draw whose coarse matrix has three exactly dependent functions: the
    # coarse term equals the pseudo-inverse form, and PCG converges to the direct solution
    from oracle.schwarz import SchwarzPreconditioner
    net = nw.fiber_network_3d(1500, 0.2, 0.01, seed=3)
    p = nw.scalar_band_problem(net, 0.25)
    free, A, _ = op.split(p)
    B = SchwarzPreconditioner(p, free, A)
    assert B.coarse.m0 - B.coarse_kept.size == 3
    r = np.random.default_rng(4).standard_normal(free.size)
    ref = _pinv_coarse_term(B, r)
    assert np.linalg.norm(B.coarse_term(r) - ref) <= 1e-8 * np.linalg.norm(ref)
    S = OracleSolver(p)
    res = S.solve(rtol=1e-10)
    import scipy.sparse.linalg as spla
    x = spla.spsolve(S.A.tocsc(), res.b)
    assert np.linalg.norm(res.x - x) <= 1e-8 * np.linalg.norm(x)


def test_structural_workload_as_written_sets_up_and_gives_zero():
    # the 20000-fibre structural network spans nothing: the clamped component alone is
    # kept, f = 0 and the Dirichlet data there are zero, so u = 0; its many sparsely
    # populated elements make coarse functions dependent (A_0 singular), which the
    # dropped functions handle
    p = nw.config3()
    S = OracleSolver(p)
    assert S.B.coarse_kept.size < S.B.coarse.m0
    res = S.solve(rtol=1e-8)
    assert res.converged and np.all(res.u == 0.0)
