"""Pins of the oracle's operator assembly and Dirichlet lifting (no GPU)."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import operator as op
from oracle.solve import OracleSolver
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


# ---------------------------------------------------------------------------
# the beam model (eq. tensile + eq. bend, Section 6.3)
# ---------------------------------------------------------------------------
def _three_node_wire():
    X = np.array([[0.5, 0.5], [0.4, 0.5], [0.6, 0.5]])
    E = np.array([[0, 1], [0, 2]], dtype=np.int64)
    AE = np.pi * nw.BEAM_RW ** 2 * nw.BEAM_E
    net = nw.Network(2, X, E, np.zeros(2, np.int8), np.ones(2), np.full(2, AE), np.zeros((2, 2)),
                     (1.0, 1.0), np.zeros(2, np.int64))
    p = nw.Problem(net, 3, "beam", np.zeros(0, np.int64), np.zeros(0), np.zeros(9), 0.5,
                   (0, 0, 0), "all", meta={"triples": nw.beam_triples(net), "r_w": nw.BEAM_RW})
    return p, AE, AE * nw.BEAM_RW ** 2 / 4.0


def test_beam_three_node_energies():
    p, AE, EI = _three_node_wire()
    assert p.meta["triples"].tolist() == [[0, 1, 2, 1]]
    K = op.assemble(p).toarray()
    g = read_golden("beam_three_nodes.txt")["energies"]
    d = 1e-3
    motions = {0: (1, 0, -d), 1: (0, 1, d), 2: (0, 2, d)}  # (node, component, displacement)
    for mid, want in g:
        node, comp, val = motions[int(mid)]
        v = np.zeros(9)
        v[3 * node + comp] = val
        scale = AE if int(mid) == 0 else EI
        assert abs(v @ K @ v - want * scale * d * d) <= 1e-12 * want * scale * d * d


def _small_beam(lateral):
    net = nw.fiber_network_2d(0, 0.05, 7, midpoint_pad=0.025, keep="boundary", total_length=40.0,
                              bias="placement" if lateral else "orientation")
    return nw.beam_problem(net, 0.25, lateral=lateral)


def test_beam_rigid_motions_are_the_kernel():
    # three translations and the in-plane rotation cost nothing; the rotations about
    # in-plane axes cost nothing on wires (pairs along one fibre), and do cost at joints
    p = _small_beam(True)
    K = op.assemble(p)
    X = p.net.coords
    n = p.net.n_nodes
    modes = []
    for a in range(3):
        m = np.zeros(3 * n)
        m[a::3] = 1.0
        modes.append(m)
    rot = np.zeros(3 * n)
    rot[0::3], rot[1::3] = -X[:, 1], X[:, 0]
    modes.append(rot)
    kmax = np.abs(K.data).max()
    for m in modes:
        assert np.abs(K @ m).max() <= 1e-10 * kmax * np.abs(m).max()
    # a single straight wire: the rotations about in-plane axes are in the kernel too
    q, _, _ = _three_node_wire()
    Kw = op.assemble(q)
    Xw = q.net.coords
    for axis in range(2):
        m = np.zeros(9)
        m[2::3] = Xw[:, 1] if axis == 0 else -Xw[:, 0]
        assert np.abs(Kw @ m).max() <= 1e-10 * np.abs(Kw.data).max()
    # and a bent wire does cost: a random motion has positive energy
    v = np.random.default_rng(0).standard_normal(3 * n)
    assert v @ (K @ v) > 0
    assert abs(K - K.T).max() <= 1e-14 * kmax


@pytest.mark.parametrize("lateral", [False, True])
def test_beam_free_block_spd_and_pcg_matches_direct(lateral):
    p = _small_beam(lateral)
    S = OracleSolver(p)
    Ad = S.A.toarray()
    np.linalg.cholesky(Ad)  # SPD once Gamma holds the wires
    res = S.solve(rtol=1e-11)
    assert np.linalg.norm(res.b - Ad @ res.x) <= 1e-11 * np.linalg.norm(res.b) * (1 + 1e-9)
    # against the dense direct solve: both are accurate to cond(A) times the rounding unit
    ev = np.linalg.eigvalsh(Ad)
    x = np.linalg.solve(Ad, res.b)
    tol = max(1e-10, 100 * ev[-1] / ev[0] * np.finfo(float).eps)
    assert np.linalg.norm(res.x - x) <= tol * np.linalg.norm(x)
    X = p.net.coords
    hi = np.nonzero(X[:, 0] >= 1.0)[0]
    np.testing.assert_allclose(res.u[3 * hi], 0.1 if lateral else 0.2)


@pytest.mark.parametrize("lateral,seed,total", [(False, 17, 60.0), (False, 3, 60.0), (True, 17, 60.0),
                                                (True, 0, 60.0)])
def test_beam_networks_have_no_free_mechanism(lateral, seed, total):
    """Networks on which, before the component prune, a fibre cluster hung from the clamped
    sides at a single node (a pin about which the in-plane bending form lets it turn): after
    beam_problem's pruning every component of the non-Dirichlet graph reaches two Dirichlet
    nodes, and K on the free dofs is positive definite."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    net = nw.fiber_network_2d(0, 0.05, seed, midpoint_pad=0.025, keep="boundary", total_length=total,
                              bias="placement" if lateral else "orientation")
    p = nw.beam_problem(net, 0.25, lateral=lateral)
    X = p.net.coords
    dmask = (X[:, 0] <= 0.0) | (X[:, 0] >= 1.0)
    E = p.net.edges
    inner = ~dmask[E[:, 0]] & ~dmask[E[:, 1]]
    n = p.net.n_nodes
    G = sp.coo_matrix((np.ones(int(inner.sum())), (E[inner, 0], E[inner, 1])), shape=(n, n))
    _, comp = connected_components(G, directed=False)
    pins = {}
    for a, b in E[dmask[E[:, 0]] ^ dmask[E[:, 1]]]:
        free_end, pin = (b, a) if dmask[a] else (a, b)
        pins.setdefault(comp[free_end], set()).add(pin)
    for c in np.unique(comp[~dmask]):
        assert len(pins.get(c, ())) >= 2, c
    _, A, _ = op.split(p, op.assemble(p))
    ev = np.linalg.eigvalsh(A.toarray())
    # positive definite, well above rounding (edges of 5e-6 to 0.05 put cond(A) near 1e13;
    # before the prune these networks had zero or negative eigenvalues of order 1e-5)
    assert ev[0] > 1e-14 * ev[-1], (ev[0], ev[-1])


def test_beam_parallel_edges_count_once():
    """Two fibres between the same two merged joints give one edge of the beam problem, so no
    bending triple pairs an edge with itself (y = z)."""
    net = nw.fiber_network_2d(0, 0.05, 6100, midpoint_pad=0.025, keep="boundary", total_length=300.0,
                              bias="orientation")
    key = np.sort(net.edges, axis=1)
    assert np.unique(key, axis=0).shape[0] < key.shape[0]   # the raw network has parallel edges
    p = nw.beam_problem(net, 0.25, lateral=False)
    key = np.sort(p.net.edges, axis=1)
    assert np.unique(key, axis=0).shape[0] == key.shape[0]
    T = p.meta["triples"]
    assert np.all((T[:, 0] != T[:, 1]) & (T[:, 0] != T[:, 2]) & (T[:, 1] != T[:, 2]))
