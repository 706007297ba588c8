"""Pins of the oracle's mesh, Q1 values, coarse dofs and Galerkin matrix (no GPU)."""
import numpy as np

from conftest import read_golden
from oracle import coarse as co
from oracle import operator as op
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
