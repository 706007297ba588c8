"""Pins of the oracle's operator assembly and Dirichlet lifting (no GPU)."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import operator as op
from paper_2207_07488_gb300 import networks as nw


def _net_from(coords, edges, cond=None, stiff=None, dirs=None, dim=None):
    coords = np.asarray(coords, float)
    edges = np.asarray(edges, np.int64)
    m = edges.shape[0]
    dim = coords.shape[1] if dim is None else dim
    cond = np.ones(m) if cond is None else np.asarray(cond, float)
    stiff = np.ones(m) if stiff is None else np.asarray(stiff, float)
    dirs = np.tile(np.eye(dim)[0], (m, 1)) if dirs is None else np.asarray(dirs, float)
    return nw.Network(dim, coords, edges, np.zeros(m, np.int8), cond, stiff, dirs,
                      tuple([1.0] * dim))


def _problem(net, ndof=1, model="scalar", dd=(), dv=()):
    return nw.Problem(net, ndof, model, np.asarray(dd, np.int64), np.asarray(dv, float),
                      np.zeros(net.n_nodes * ndof), 0.5, (0,) * ndof)


def test_three_node_hand_computed():
    g = read_golden("three_node_scalar.txt")
    E = g["edges"]
    net = _net_from(g["coords"], E[:, :2].astype(int), cond=E[:, 2])
    K = op.assemble(_problem(net)).toarray()
    np.testing.assert_allclose(K, g["K"], rtol=0, atol=1e-15)


def test_truss_edge_hand_computed():
    g = read_golden("truss_edge.txt")
    blk = g["block"]
    net = _net_from([[0, 0, 0], [0.5, 0.5, 0]], [[0, 1]], stiff=[2.0], dirs=[[0.6, 0.8, 0.0]])
    K = op.assemble(_problem(net, 3, "truss3")).toarray()
    ref = np.block([[blk, -blk], [-blk, blk]])
    np.testing.assert_allclose(K, ref, rtol=0, atol=1e-14)


def test_laplacian_symmetric_zero_rowsum_psd():
    p = nw.config1()
    K = op.assemble(p)
    assert abs(K - K.T).max() == 0.0
    rs = np.abs(K @ np.ones(K.shape[0]))
    assert rs.max() <= 1e-12 * abs(K).max()
    # kernel: the constants (eq. 2.2); PSD on a small network
    small = nw.fiber_network_2d(60, 0.3, seed=5)
    Ks = op.assemble(nw.scalar_band_problem(small, 0.5)).toarray()
    ev = np.linalg.eigvalsh(Ks)
    assert ev[0] > -1e-10 * ev[-1]


def test_truss_kernel_is_translations():
    net = nw.fiber_network_3d(300, 0.3, 0.03, seed=11, keep="clamped_x")
    p = nw.truss_band_problem(net, 0.5)
    K = op.assemble(p)
    n = net.n_nodes
    for a in range(3):
        t = np.zeros(3 * n)
        t[a::3] = 1.0
        assert np.abs(K @ t).max() <= 1e-10 * abs(K).max()
    # a rotation is not in the kernel once the lateral term is present
    X = net.coords
    rot = np.zeros(3 * n)
    rot[0::3] = -X[:, 1]
    rot[1::3] = X[:, 0]
    assert rot @ (K @ rot) > 1e-6 * abs(K).max()


def test_lifting_chain_closed_form():
    # chain 0-1-2 with unit conductances, u(0) = 0, u(2) = 1: the free value is 1/2
    net = _net_from([[0, 0], [0.5, 0], [1, 0]], [[0, 1], [1, 2]])
    p = _problem(net, dd=[0, 2], dv=[0.0, 1.0])
    free, A, KID = op.split(p)
    b = op.lifted_rhs(p, p.f, p.dirichlet_vals, free, KID)
    assert free.tolist() == [1]
    assert np.allclose(A.toarray(), [[2.0]]) and np.allclose(b, [1.0])
    u = op.expand(p, free, np.linalg.solve(A.toarray(), b), p.dirichlet_vals)
    np.testing.assert_allclose(u, [0.0, 0.5, 1.0])


def test_free_block_spd():
    p = nw.config1()
    free, A, _ = op.split(p)
    np.linalg.cholesky(A.toarray())   # raises if not SPD (Example 3.2)
