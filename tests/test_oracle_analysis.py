"""Pins of the oracle's network analysis (Section 3.2 homogeneity, Lemma 3.5 connectivity):
node masses and box masses on a regular grid by hand, lambda_2 of L u = lambda M u on a path
and a cycle against their closed forms, the breadth-first connecting subgraph on small
hand-made networks, and the largest component."""
from dataclasses import replace

import numpy as np
import pytest

from oracle.analysis import (connecting_subgraph, homogeneity, lambda2, largest_component,
                             node_mass)
from paper_2207_07488_gb300 import networks as nw


def _net(coords, edges):
    """A scalar network from coordinates and an edge list (conductances unused here)."""
    coords = np.asarray(coords, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.int64)
    base = nw.grid_heat_problem(2, 0.5).net
    m = edges.shape[0]
    return replace(base, coords=coords, edges=edges, kind=np.zeros(m, dtype=base.kind.dtype),
                   cond=np.ones(m), stiff=np.ones(m), dirs=np.zeros((m, coords.shape[1])),
                   fiber=None)


def test_node_and_box_masses_on_a_grid():
    # the (2^3+1)^2 grid of spacing h = 1/8: m = 2h inside, 3h/2 on a side, h at a corner
    net = nw.grid_heat_problem(3, 0.25).net
    h = 1.0 / 8
    m = node_mass(net)
    X = net.coords
    on = (np.isclose(X, 0.0) | np.isclose(X, 1.0)).sum(axis=1)
    np.testing.assert_allclose(m[on == 0], 2 * h)
    np.testing.assert_allclose(m[on == 1], 1.5 * h)
    np.testing.assert_allclose(m[on == 2], h)
    # R^-1 = 4: cells of side 1/2, half-open (closed at the domain's upper edges).  The lower
    # left cell holds x, y in {0, .., 3} h: one corner, 6 side nodes, 9 inner nodes; the upper
    # right cell holds {4, .., 8} h: 25 nodes, 1 corner, 8 side nodes, 16 inner nodes
    vals, sigma, rho = homogeneity(net, 4)
    side2 = 0.25
    assert vals[0] == pytest.approx((h + 6 * 1.5 * h + 9 * 2 * h) / side2)
    assert vals[3] == pytest.approx((h + 8 * 1.5 * h + 16 * 2 * h) / side2)
    assert sigma == pytest.approx(vals.max() / vals.min()) and rho == pytest.approx(vals.min())
    # the masses sum to the total edge length: 2 * 8 * 9 edges of length h
    assert vals.sum() * side2 == pytest.approx(2 * 8 * 9 * h)


@pytest.mark.parametrize("n,h", [(5, 0.1), (9, 0.03), (17, 0.5)])
def test_lambda2_closed_forms(n, h):
    # a uniform path with lumped masses: lambda_2 = (4 / h^2) sin^2(pi / (2 (n - 1)))
    X = np.stack([np.arange(n) * h, np.zeros(n)], axis=1)
    path = _net(X, [[i, i + 1] for i in range(n - 1)])
    got = lambda2(path, np.arange(n - 1))
    assert got == pytest.approx(4 / h ** 2 * np.sin(np.pi / (2 * (n - 1))) ** 2, rel=1e-10)
    # a regular n-gon of side h: lambda_2 = (4 / h^2) sin^2(pi / n)
    r = h / (2 * np.sin(np.pi / n))
    t = 2 * np.pi * np.arange(n) / n
    ring = _net(np.stack([r * np.cos(t), r * np.sin(t)], axis=1), [[i, (i + 1) % n] for i in range(n)])
    got = lambda2(ring, np.arange(n))
    assert got == pytest.approx(4 / h ** 2 * np.sin(np.pi / n) ** 2, rel=1e-10)


def test_lambda2_large_subgraph_uses_shift_invert():
    # above the dense size the shift-and-invert branch runs: a path of 2001 nodes
    n, h = 2001, 1e-3
    X = np.stack([np.arange(n) * h, np.zeros(n)], axis=1)
    path = _net(X, [[i, i + 1] for i in range(n - 1)])
    got = lambda2(path, np.arange(n - 1))
    assert got == pytest.approx(4 / h ** 2 * np.sin(np.pi / (2 * (n - 1))) ** 2, rel=1e-8)


def _two_pieces():
    """In the box [0, 0.5)^2 two pieces, {0, 1} and {2, 3}.  The edges with an endpoint in the
    box reach nodes 4 and 5 just outside it (so G' starts as {0, 1, 4} and {2, 3, 5}); the
    pieces are joined by the edge 4-5, by the longer path 4-6-7-5, and by 4-8-5 through a node
    far outside the ring."""
    X = [[0.1, 0.1], [0.4, 0.1], [0.4, 0.4], [0.1, 0.4], [0.55, 0.1], [0.55, 0.4],
         [0.58, 0.2], [0.58, 0.3], [0.9, 0.25]]
    E = [[0, 1], [2, 3], [1, 4], [5, 2], [4, 5], [4, 6], [6, 7], [7, 5], [4, 8], [8, 5]]
    return _net(X, E)


def test_connecting_subgraph_takes_the_shortest_path_in_the_ring():
    net = _two_pieces()
    ids = connecting_subgraph(net, np.zeros(2), np.full(2, 0.5), 0.1)
    # the four edges with an endpoint in the box and the one-edge link 4-5 (not the longer
    # path 4-6-7-5, not the way through node 8 beyond the ring)
    assert sorted(ids.tolist()) == [0, 1, 2, 3, 4]
    # without the short link the breadth-first search takes the three-edge path
    drop = _net(net.coords, np.delete(net.edges, 4, axis=0))
    ids = connecting_subgraph(drop, np.zeros(2), np.full(2, 0.5), 0.1)
    assert sorted(ids.tolist()) == [0, 1, 2, 3, 4, 5, 6]


def test_connecting_subgraph_fails_without_a_path_in_the_ring():
    net = _two_pieces()
    # a ring of width 0.02 leaves nodes 4 and 5 outside it: no joining edge is allowed
    assert connecting_subgraph(net, np.zeros(2), np.full(2, 0.5), 0.02) is None


def test_connecting_subgraph_keeps_edges_that_leave_the_ring():
    # an edge from a box node to a node beyond the ring is kept (it has an endpoint in the box)
    net = _net([[0.2, 0.2], [0.3, 0.2], [0.9, 0.2]], [[0, 1], [1, 2]])
    ids = connecting_subgraph(net, np.zeros(2), np.full(2, 0.5), 0.05)
    assert sorted(ids.tolist()) == [0, 1]


def test_largest_component():
    net = _two_pieces()
    extra = _net(np.vstack([net.coords, [[0.8, 0.1], [0.9, 0.1]]]),
                 np.vstack([net.edges, [[9, 10]]]))
    big = largest_component(extra)
    assert big.n_nodes == 9 and big.n_edges == net.n_edges
    np.testing.assert_array_equal(big.coords, net.coords)
