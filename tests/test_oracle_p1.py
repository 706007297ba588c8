"""Pins of the oracle's P1 coarse space on simplices (Remark 2.1; the Kuhn triangulation of
the box mesh).

The point location and its tie-break are checked against a brute-force search over
explicitly built simplices (barycentric coordinates from linear solves, the lowest element
number that holds the point); the basis values against those barycentric coordinates; the
Galerkin matrix on a grid network against the textbook P1 stiffness stencil of right
triangles (and the Q1 one against the bilinear stencil, which tells the two apart); the
element patches against brute force; and a solve."""
import itertools
from dataclasses import replace

import numpy as np
import pytest

from oracle import operator as oop
from oracle.coarse import CoarseSpace, host_simplices, p1_values
from oracle.schwarz import star_dofs
from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw


def explicit_elements(nH, h):
    """(box multi-index, permutation, vertex coordinates (d+1, d), vertex corner bits) of
    every element, in element-number order: boxes linearly with axis 0 fastest, the
    simplices of a box by the lexicographic order of the permutation."""
    d = len(nH)
    out = []
    for rev in itertools.product(*[range(n) for n in reversed(nH)]):
        box = np.array(rev[::-1])
        for perm in itertools.permutations(range(d)):
            verts = [box * h]
            bits = [0]
            cur = box.astype(float).copy()
            b = 0
            for a in perm:
                cur = cur.copy()
                cur[a] += 1
                b |= 1 << a
                verts.append(cur * h)
                bits.append(b)
            out.append((box, perm, np.array(verts), bits))
    return out


def barycentric(verts, x):
    d = x.size
    M = np.vstack([verts.T, np.ones(d + 1)])
    return np.linalg.solve(M, np.append(x, 1.0))


def brute_force(elements, x, tol=1e-12):
    for j, (box, perm, verts, bits) in enumerate(elements):
        lam = barycentric(verts, x)
        if np.all(lam >= -tol):
            return j, box, perm, lam, bits
    raise AssertionError(f"no element holds {x}")


def _points(nH, h, rng, n_random=150):
    d = len(nH)
    pts = [rng.uniform(0, 1, size=d) * np.array(nH) * h for _ in range(n_random)]
    # points on box faces, edges, corners and the simplices' shared faces (t_a = t_b), where
    # the mesh width is a power of two so that the ties are exact in floating point
    if all(n & (n - 1) == 0 for n in nH):
        grid = [np.arange(0, 4 * n + 1) * (hh / 4) for n, hh in zip(nH, h)]
        for p in itertools.product(*grid):
            pts.append(np.array(p))
    return np.array(pts)


@pytest.mark.parametrize("nH", [(4, 2), (3, 3), (2, 2, 2), (3, 1, 2), (4, 2, 1)])
def test_point_location_and_values_against_brute_force(nH):
    d = len(nH)
    h = np.array([1.0 / n for n in nH])
    rng = np.random.default_rng(len(nH) * 10 + nH[0])
    X = _points(nH, h, rng)
    els = explicit_elements(nH, h)
    e, pidx, t = host_simplices(X, np.ones(d), nH)
    W, V = p1_values(t, pidx, d)
    perms = list(itertools.permutations(range(d)))
    for r in range(X.shape[0]):
        j, box, perm, lam, bits = brute_force(els, X[r])
        assert tuple(e[r]) == tuple(box), (X[r], e[r], box)
        assert perms[pidx[r]] == perm, (X[r], perms[pidx[r]], perm)
        Wb = np.zeros(2 ** d)
        Wb[bits] = lam
        np.testing.assert_allclose(W[r], Wb, rtol=0, atol=1e-12)
        assert set(np.nonzero(V[r])[0]) == set(bits)


@pytest.mark.parametrize("nH", [(3, 2), (2, 2, 2)])
def test_simplices_tile_the_boxes(nH):
    d = len(nH)
    h = np.array([1.0 / n for n in nH])
    els = explicit_elements(nH, h)
    vol = np.prod(h)
    for box, perm, verts, bits in els:
        v = abs(np.linalg.det(verts[1:] - verts[0])) / np.prod(np.arange(1, d + 1))
        assert abs(v - vol / np.prod(np.arange(1, d + 1))) < 1e-14
    rng = np.random.default_rng(5)
    for x in rng.uniform(0, 1, size=(200, d)):   # interior points lie in exactly one simplex
        inside = [j for j, (_, _, verts, _) in enumerate(els) if np.all(barycentric(verts, x) > 1e-12)]
        assert len(inside) == 1


@pytest.mark.parametrize("nH", [(4, 2), (2, 2, 2)])
def test_partition_of_unity_affine_reproduction_and_continuity(nH):
    d = len(nH)
    h = np.array([1.0 / n for n in nH])
    rng = np.random.default_rng(11)
    X = _points(nH, h, rng, 300)
    e, pidx, t = host_simplices(X, np.ones(d), nH)
    W, _ = p1_values(t, pidx, d)
    corners = np.array([[(c >> a) & 1 for a in range(d)] for c in range(2 ** d)])
    A = rng.normal(size=d)
    f = lambda y: 0.7 + y @ A  # noqa: E731
    val = sum(W[:, c] * f((e + corners[c]) * h) for c in range(2 ** d))
    np.testing.assert_allclose(W.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(val, f(X), atol=1e-13)
    assert np.all(W >= -1e-15)
    # continuity: a random nodal vector interpolated from every element that holds a point
    els = explicit_elements(nH, h)
    zc = {}
    for x in X[:80]:
        vals = []
        for box, perm, verts, bits in els:
            lam = barycentric(verts, x)
            if np.all(lam >= -1e-12):
                vals.append(sum(lam[j] * zc.setdefault(tuple(np.round(verts[j] / h).astype(int)), rng.normal())
                                for j in range(d + 1)))
        assert max(vals) - min(vals) < 1e-12


def test_box_centre_value():
    # the centre of a square lies on the shared diagonal t_0 = t_1: half at the two ends of
    # the diagonal, nothing at the other two corners (Q1 would give a quarter to each)
    e, pidx, t = host_simplices(np.array([[0.125, 0.125]]), np.ones(2), (4, 4))
    W, V = p1_values(t, pidx, 2)
    np.testing.assert_allclose(W[0], [0.5, 0.0, 0.0, 0.5], atol=1e-15)


@pytest.mark.parametrize("k", [5, 6])
def test_galerkin_stencils_on_a_grid(k):
    """On the (2^k+1)^2 unit-conductance grid, delta * A_0 (delta = 2^-k the grid spacing) at an
    interior mesh node: P1 on the Kuhn triangles gives the right-triangle stiffness stencil
    (4 at the centre, -1 along the axes, 0 on the diagonals) exactly; Q1 gives the bilinear
    stencil (8/3 and -1/3 at all eight neighbours) up to O(delta / H)."""
    p = nw.grid_heat_problem(k, 0.25)
    delta = 2.0 ** -k
    got = {}
    for space in ("p1", "q1"):
        q = replace(p, coarse=space)
        K = oop.assemble(q)
        free, A, _ = oop.split(q, K)
        C = CoarseSpace(q, free, A)
        idx = C.coarse_index
        c = idx[2 + 5 * 2, 0]
        got[space] = {(dx, dy): C.A0[c, idx[(2 + dx) + 5 * (2 + dy), 0]] * delta
                      for dx in (-1, 0, 1) for dy in (-1, 0, 1)}
    for (dx, dy), v in got["p1"].items():
        want = 4.0 if (dx, dy) == (0, 0) else (-1.0 if dx * dy == 0 else 0.0)
        assert abs(v - want) < 1e-12, ((dx, dy), v)
    for (dx, dy), v in got["q1"].items():
        want = 8.0 / 3.0 if (dx, dy) == (0, 0) else -1.0 / 3.0
        assert abs(v - want) < 4 * delta / 0.25, ((dx, dy), v)


def test_element_patches_against_brute_force():
    nH = (3, 2)
    h = np.array([1.0 / 3, 0.5])
    rng = np.random.default_rng(3)
    X = _points(nH, h, rng, 120)
    e, pidx, t = host_simplices(X, np.ones(2), nH)
    W, V = p1_values(t, pidx, 2)
    els = explicit_elements(nH, h)
    host_vertices = []
    for x in X:
        j, box, perm, lam, bits = brute_force(els, x)
        host_vertices.append({tuple(box + np.array([(b >> a) & 1 for a in range(2)])) for b in bits})
    for k in itertools.product(range(nH[0] + 1), range(nH[1] + 1)):
        S = set(star_dofs(e, k, nH, None, V).tolist())
        want = {r for r in range(X.shape[0]) if tuple(k) in host_vertices[r]}
        assert S == want, k
        Ssup = set(star_dofs(e, k, nH, W, None).tolist())
        assert Ssup <= S   # the support of phi_k lies inside its element patch


@pytest.mark.parametrize("patch", ["support", "element"])
def test_two_level_solve_with_p1(patch):
    p = replace(nw.grid_heat_problem(5, 0.25), coarse="p1", patch=patch)
    S = OracleSolver(p)
    r = S.solve(rtol=1e-10, maxit=200)
    assert r.converged and r.iters < 40
    b = S.rhs()
    assert np.linalg.norm(S.A @ r.x - b) <= 1e-10 * np.linalg.norm(b) * 1.01
