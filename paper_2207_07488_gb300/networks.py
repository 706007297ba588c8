"""Seeded synthetic spatial networks and problem data.

This module only builds inputs: node coordinates, edges with their material
coefficients, Dirichlet dof sets and values, right-hand sides and the coarse
mesh parameters.  It holds none of the solver's arithmetic (no operator
assembly, no preconditioner, no Krylov iteration); the CUDA library and the CPU
oracle each assemble K from these edge lists on their own.

Networks follow the paper's setting (Section 2.1): a graph whose nodes are
points of the closed box Omega = [0, l_1] x ... x [0, l_d] and whose edges join
adjacent nodes.  The fiber generators follow the construction of Section 6.1:
straight fibers placed at random and clipped to the box, a node wherever two
fibers meet, nodes merged below a length tolerance along each fiber, and
components without a Dirichlet node removed.  Per-edge coefficients:

* scalar diffusion: conductance 1/length on fiber segments, 10 on contacts;
* structural (3 dofs per node): coefficient EA/L_eff and unit direction n per
  edge, EA = 1 on fibers and 10 on contacts, L_eff = max(dist, delta/10) on
  contacts; a contact of zero length takes n = d1 x d2 of its two fibers.

Every generator is a pure function of its arguments and seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

FIBER, CONTACT = 0, 1
STAR_INTERIOR, STAR_ALL = "interior", "all"
PATCH_ELEMENT, PATCH_SUPPORT = "element", "support"
COARSE_Q1, COARSE_P1 = "q1", "p1"


def face_bit(axis: int, side: int) -> int:
    """Bit of a Dirichlet face: side 0 is x_axis = 0, side 1 is x_axis = l_axis."""
    return 1 << (2 * axis + side)


@dataclass
class Network:
    """A spatial network: nodes in a box and edges with coefficients."""

    dim: int
    coords: np.ndarray          # (n_nodes, dim) float64
    edges: np.ndarray           # (n_edges, 2) int64, i != j
    kind: np.ndarray            # (n_edges,) int8: FIBER or CONTACT
    cond: np.ndarray            # (n_edges,) float64 scalar conductance
    stiff: np.ndarray           # (n_edges,) float64 structural coefficient EA/L_eff
    dirs: np.ndarray            # (n_edges, dim) float64 unit edge direction
    domain: tuple = (1.0, 1.0)  # (l_1, ..., l_d)
    fiber: np.ndarray | None = None  # (n_edges,) int64: the fibre of a fibre edge, -1 for contacts

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])


@dataclass
class Problem:
    """A linear problem (K u, v) = (f, v) on a network with Dirichlet data.

    Dofs are numbered node-major: dof = ndof * node + component.  ``model`` is
    "scalar" (edge weights ``net.cond``) or "truss3" (3x3 edge blocks built
    from ``net.stiff`` and ``net.dirs``).  ``gamma_faces[c]`` is the bitmask of
    box faces on which component c is Dirichlet (the coarse space drops the
    mesh nodes lying on them).  ``star_set`` picks the mesh nodes that carry a
    star (the interior ones or all) and ``patch`` the nodes a star holds:
    "element" (every node whose half-open host element touches the star's mesh
    node) or "support" (only the nodes where that mesh node's Q1 basis
    function is nonzero, which leaves out nodes on the outer boundary of the
    patch).  ``coarse`` picks the coarse space: Q1 on the box mesh (Section 2.3) or
    P1 on the simplices of its Kuhn triangulation (Remark 2.1).
    """

    net: Network
    ndof: int
    model: str
    dirichlet_dofs: np.ndarray      # sorted int64
    dirichlet_vals: np.ndarray      # float64, same length
    f: np.ndarray                   # (n_nodes*ndof,) float64; Dirichlet entries ignored
    H: float
    gamma_faces: tuple
    star_set: str = STAR_INTERIOR
    name: str = ""
    meta: dict = field(default_factory=dict)
    patch: str = PATCH_ELEMENT
    coarse: str = COARSE_Q1         # Q1 on the boxes, or P1 on their Kuhn simplices (Remark 2.1)

    @property
    def n_dof(self) -> int:
        return self.net.n_nodes * self.ndof

    @property
    def nH(self) -> tuple:
        return tuple(int(round(l / self.H)) for l in self.net.domain)


# ----------------------------------------------------------------------------
# geometry helpers
# ----------------------------------------------------------------------------

def _clip_to_box(c, d, half, box):
    """Clip segments c + t d, t in [-half, half], to [0, box]; mask of non-empty ones."""
    t0 = np.full(c.shape[0], -half)
    t1 = np.full(c.shape[0], half)
    for ax in range(c.shape[1]):
        da = d[:, ax]
        nz = np.abs(da) > 0
        safe = np.where(nz, da, 1.0)
        lo = np.where(nz, (0.0 - c[:, ax]) / safe, -np.inf)
        hi = np.where(nz, (box[ax] - c[:, ax]) / safe, np.inf)
        # an axis-parallel fiber outside the slab is empty
        out = ~nz & ((c[:, ax] < 0.0) | (c[:, ax] > box[ax]))
        t0 = np.where(out, np.inf, np.maximum(t0, np.minimum(lo, hi)))
        t1 = np.minimum(t1, np.maximum(lo, hi))
    ok = t1 > t0
    t0 = np.where(ok, t0, 0.0)
    t1 = np.where(ok, t1, 0.0)
    a = np.clip(c + t0[:, None] * d, 0.0, box)
    b = np.clip(c + t1[:, None] * d, 0.0, box)
    return a, b, ok


def segment_closest(p1, q1, p2, q2):
    """Closest points of segment pairs [p1,q1] and [p2,q2] (vectorised).

    Minimises |p1 + s d1 - p2 - t d2|^2 over s, t in [0, 1]: the stationary
    point of the quadratic, clamped, then re-optimised along the clamped
    parameter.  Returns (s, t, dist).
    """
    d1 = q1 - p1
    d2 = q2 - p2
    r = p1 - p2
    a = np.einsum("ij,ij->i", d1, d1)
    e = np.einsum("ij,ij->i", d2, d2)
    f = np.einsum("ij,ij->i", d2, r)
    c = np.einsum("ij,ij->i", d1, r)
    b = np.einsum("ij,ij->i", d1, d2)
    den = a * e - b * b
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(den > 1e-14 * a * e, np.clip((b * f - c * e) / den, 0.0, 1.0), 0.0)
        t = (b * s + f) / e
        lo = t < 0.0
        hi = t > 1.0
        s = np.where(lo, np.clip(-c / a, 0.0, 1.0), s)
        s = np.where(hi, np.clip((b - c) / a, 0.0, 1.0), s)
        t = np.clip(t, 0.0, 1.0)
    P = p1 + s[:, None] * d1
    Q = p2 + t[:, None] * d2
    return s, t, np.linalg.norm(P - Q, axis=1)


def _segment_cross_2d(p1, q1, p2, q2):
    """Crossing parameters of 2D segment pairs and the mask of pairs that cross."""
    d1 = q1 - p1
    d2 = q2 - p2
    w = p2 - p1
    den = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    ok = np.abs(den) > 1e-15
    safe = np.where(ok, den, 1.0)
    s = (w[:, 0] * d2[:, 1] - w[:, 1] * d2[:, 0]) / safe
    t = (w[:, 0] * d1[:, 1] - w[:, 1] * d1[:, 0]) / safe
    hit = ok & (s >= 0.0) & (s <= 1.0) & (t >= 0.0) & (t <= 1.0)
    return s, t, hit


def _keep_fn(keep):
    if keep == "dirichlet_x":
        return lambda X: (X[:, 0] < 0.01) | (X[:, 0] > 0.99)
    if keep == "clamped_x":
        return lambda X: X[:, 0] < 0.01
    if keep == "boundary":
        return lambda X: np.any((X <= 0.0) | (X >= 1.0), axis=1)
    raise ValueError(keep)


def _build(dim, pts, fib, pos, joins, contacts, merge_tol, keep_mask, fiber_dir,
           contact_cond, delta):
    """Turn fiber incidences into a network.

    Point k is an incidence of fiber fib[k] at arc position pos[k].  ``joins``
    are point pairs that are one node (a 2D crossing seen from both fibers);
    ``contacts`` are point pairs joined by a contact edge.  Points closer than
    ``merge_tol`` along one fiber become one node, placed at the member with
    the smallest point id.
    """
    n_pts = pts.shape[0]
    order = np.lexsort((np.arange(n_pts), pos, fib))
    fs, ps = fib[order], pos[order]
    same = (fs[1:] == fs[:-1]) & (ps[1:] - ps[:-1] < merge_tol)
    mi = np.concatenate([order[:-1][same], joins[:, 0]])
    mj = np.concatenate([order[1:][same], joins[:, 1]])
    G = sp.coo_matrix((np.ones(mi.size), (mi, mj)), shape=(n_pts, n_pts))
    n_lab, lab = connected_components(G, directed=False)
    rep = np.full(n_lab, n_pts, dtype=np.int64)
    np.minimum.at(rep, lab, np.arange(n_pts))
    node_pos = pts[rep]
    # fiber segments between consecutive distinct nodes of one fiber
    na, nb = lab[order[:-1]], lab[order[1:]]
    fe = (fs[1:] == fs[:-1]) & (na != nb)
    ei, ej = [na[fe]], [nb[fe]]
    fids = [fs[1:][fe].astype(np.int64)]
    kinds = [np.full(int(fe.sum()), FIBER, np.int8)]
    cfib = np.zeros((0, 2), np.int64)
    if contacts.size:
        ci, cj = lab[contacts[:, 0]], lab[contacts[:, 1]]
        ok = ci != cj
        ei.append(ci[ok])
        ej.append(cj[ok])
        fids.append(np.full(int(ok.sum()), -1, np.int64))
        kinds.append(np.full(int(ok.sum()), CONTACT, np.int8))
        cfib = np.stack([fib[contacts[ok, 0]], fib[contacts[ok, 1]]], axis=1)
    ei = np.concatenate(ei)
    ej = np.concatenate(ej)
    fid = np.concatenate(fids)
    kind = np.concatenate(kinds)
    # keep components that reach the Dirichlet region
    A = sp.coo_matrix((np.ones(ei.size), (ei, ej)), shape=(n_lab, n_lab))
    n_comp, comp = connected_components(A, directed=False)
    used = np.zeros(n_lab, bool)
    used[ei] = True
    used[ej] = True
    good_comp = np.zeros(n_comp, bool)
    good_comp[comp[used & keep_mask(node_pos)]] = True
    keep = used & good_comp[comp]
    new_id = -np.ones(n_lab, np.int64)
    new_id[keep] = np.arange(int(keep.sum()))
    coords = node_pos[keep]
    ek = keep[ei]
    E = np.stack([new_id[ei[ek]], new_id[ej[ek]]], axis=1)
    kind = kind[ek]
    fid = fid[ek]
    n_fiber_edges = int((kind == FIBER).sum())
    cfib = cfib[ek[ek.size - cfib.shape[0]:]] if cfib.shape[0] else cfib
    vec = coords[E[:, 1]] - coords[E[:, 0]]
    dist = np.linalg.norm(vec, axis=1)
    isf = kind == FIBER
    isc = ~isf
    cond = np.empty(E.shape[0])
    stiff = np.empty(E.shape[0])
    cond[isf] = 1.0 / np.maximum(dist[isf], 1e-300)
    stiff[isf] = 1.0 / np.maximum(dist[isf], 1e-300)
    cond[isc] = contact_cond
    stiff[isc] = 10.0 / np.maximum(dist[isc], delta / 10.0)
    dirs = np.zeros_like(vec)
    long_ = dist > 1e-12
    dirs[long_] = vec[long_] / dist[long_, None]
    short = np.nonzero(~long_)[0]
    if short.size:
        for k in short:
            if kind[k] == CONTACT and dim == 3:
                f1, f2 = cfib[k - n_fiber_edges]
                nv = np.cross(fiber_dir[f1], fiber_dir[f2])
                nn = np.linalg.norm(nv)
                dirs[k] = nv / nn if nn > 0 else np.eye(3)[0]
            else:
                dirs[k] = np.eye(dim)[0]
    return coords, E.astype(np.int64), kind, cond, stiff, dirs, fid


# ----------------------------------------------------------------------------
# generators
# ----------------------------------------------------------------------------

def _draw_fibres(rng, count, pad, bias):
    """Midpoints and angles of `count` fibres.  bias None: uniform midpoints in
    [-pad, 1+pad]^2 and uniform angles; "orientation": angles concentrated about the
    x_1 axis (the doubled angle von Mises with concentration 2); "placement": the x_1 of
    the midpoints arcsine-distributed over [-pad, 1+pad] (denser near x_1 = 0 and 1).
    The paper (Section 6.1) names the two biases without their distributions; these are
    stand-ins of the same kind."""
    if bias == "placement":
        c = np.stack([-pad + (1.0 + 2.0 * pad) * rng.beta(0.5, 0.5, size=count),
                      rng.uniform(-pad, 1.0 + pad, size=count)], axis=1)
    else:
        c = rng.uniform(-pad, 1.0 + pad, size=(count, 2))
    if bias == "orientation":
        th = 0.5 * rng.vonmises(0.0, 2.0, size=count)
    else:
        th = rng.uniform(0.0, np.pi, size=count)
    return c, th


def fiber_network_2d(n_fibers: int, length: float, seed: int, merge_tol: float | None = None,
                     midpoint_pad: float = 0.0, keep: str = "dirichlet_x",
                     total_length: float | None = None, bias: str | None = None) -> Network:
    """2D fiber network: straight fibers with a node at every crossing and end.

    Midpoints uniform in [-pad, 1+pad]^2, angles uniform in [0, pi), fibers
    clipped to the unit square; each pairwise crossing is a node shared by
    both fibers; nodes closer than ``merge_tol`` (default length*1e-4) along a
    fiber are merged (Section 6.1).  With ``total_length`` set, fibers are
    drawn until their clipped length reaches it and ``n_fibers`` is ignored.
    ``bias`` ("orientation" or "placement") draws the biased networks (see
    _draw_fibres).
    """
    rng = np.random.default_rng(seed)
    box = np.array([1.0, 1.0])
    if merge_tol is None:
        merge_tol = length * 1e-4
    if total_length is None:
        c, th = _draw_fibres(rng, n_fibers, midpoint_pad, bias)
        d = np.stack([np.cos(th), np.sin(th)], axis=1)
        a, b, ok = _clip_to_box(c, d, length / 2, box)
        a, b, d = a[ok], b[ok], d[ok]
    else:
        As, Bs, Ds, tot = [], [], [], 0.0
        while tot < total_length:
            c, th = _draw_fibres(rng, 1, midpoint_pad, bias)
            dd = np.stack([np.cos(th), np.sin(th)], axis=1)
            a1, b1, ok = _clip_to_box(c, dd, length / 2, box)
            if ok[0] and np.linalg.norm(b1 - a1) > 0:
                As.append(a1)
                Bs.append(b1)
                Ds.append(dd)
                tot += float(np.linalg.norm(b1 - a1))
        a, b, d = np.concatenate(As), np.concatenate(Bs), np.concatenate(Ds)
    seg = np.linalg.norm(b - a, axis=1)
    nz = seg > 0
    a, b, d, seg = a[nz], b[nz], d[nz], seg[nz]
    nf = a.shape[0]
    tree = cKDTree(0.5 * (a + b))
    pairs = tree.query_pairs(r=length, output_type="ndarray")
    if pairs.size == 0:
        pairs = np.zeros((0, 2), np.int64)
    i, j = pairs[:, 0], pairs[:, 1]
    s, t, hit = _segment_cross_2d(a[i], b[i], a[j], b[j])
    i, j, s, t = i[hit], j[hit], s[hit], t[hit]
    xp = a[i] + s[:, None] * (b[i] - a[i])
    nx = i.size
    pts = np.concatenate([a, b, xp, xp], axis=0)
    fib = np.concatenate([np.arange(nf), np.arange(nf), i, j])
    pos = np.concatenate([np.zeros(nf), seg, s * seg[i], t * seg[j]])
    joins = np.stack([2 * nf + np.arange(nx), 2 * nf + nx + np.arange(nx)], axis=1)
    coords, E, kind, cond, stiff, dirs, fid = _build(
        2, pts, fib, pos, joins, np.zeros((0, 2), np.int64), merge_tol, _keep_fn(keep),
        d, 10.0, 0.0)
    return Network(2, coords, E, kind, cond, stiff, dirs, (1.0, 1.0), fid)


def fiber_network_3d(n_fibers: int, length: float, contact_dist: float, seed: int,
                     merge_tol: float | None = None, keep: str = "dirichlet_x",
                     chunk: int = 2_000_000) -> Network:
    """3D fiber network with contact edges.

    Fibers of the given length with midpoints uniform in the unit cube and
    isotropic directions (normalised Gaussian vectors) are clipped to the
    cube.  Two fibers whose segment distance is below ``contact_dist`` are in
    contact: the two closest points become nodes on their fibers, joined by a
    contact edge.  Nodes closer than ``merge_tol`` (default length*1e-4) along
    a fiber are merged, so a contact at a fiber end reuses the end node.
    """
    rng = np.random.default_rng(seed)
    box = np.array([1.0, 1.0, 1.0])
    if merge_tol is None:
        merge_tol = length * 1e-4
    c = rng.uniform(0.0, 1.0, size=(n_fibers, 3))
    g = rng.standard_normal(size=(n_fibers, 3))
    d = g / np.linalg.norm(g, axis=1, keepdims=True)
    a, b, ok = _clip_to_box(c, d, length / 2, box)
    seg = np.linalg.norm(b - a, axis=1)
    ok &= seg > 0
    a, b, d, seg = a[ok], b[ok], d[ok], seg[ok]
    nf = a.shape[0]
    tree = cKDTree(0.5 * (a + b))
    pairs = tree.query_pairs(r=length + contact_dist, output_type="ndarray")
    if pairs.size == 0:
        pairs = np.zeros((0, 2), np.int64)
    I, J, S, T = [], [], [], []
    for k0 in range(0, pairs.shape[0], chunk):
        i, j = pairs[k0:k0 + chunk, 0], pairs[k0:k0 + chunk, 1]
        s, t, dist = segment_closest(a[i], b[i], a[j], b[j])
        hit = dist < contact_dist
        I.append(i[hit]); J.append(j[hit]); S.append(s[hit]); T.append(t[hit])
    i = np.concatenate(I) if I else np.zeros(0, np.int64)
    j = np.concatenate(J) if J else np.zeros(0, np.int64)
    s = np.concatenate(S) if S else np.zeros(0)
    t = np.concatenate(T) if T else np.zeros(0)
    nc = i.size
    P = a[i] + s[:, None] * (b[i] - a[i])
    Q = a[j] + t[:, None] * (b[j] - a[j])
    pts = np.concatenate([a, b, P, Q], axis=0)
    fib = np.concatenate([np.arange(nf), np.arange(nf), i, j])
    pos = np.concatenate([np.zeros(nf), seg, s * seg[i], t * seg[j]])
    contacts = np.stack([2 * nf + np.arange(nc), 2 * nf + nc + np.arange(nc)], axis=1)
    coords, E, kind, cond, stiff, dirs, fid = _build(
        3, pts, fib, pos, np.zeros((0, 2), np.int64), contacts, merge_tol, _keep_fn(keep),
        d, 10.0, contact_dist)
    return Network(3, coords, E, kind, cond, stiff, dirs, (1.0, 1.0, 1.0), fid)


def grid_network_2d(k: int) -> Network:
    """(2^k + 1)^2 grid on the unit square, edges between axis neighbours.

    Node (a, b) has id a + n*b and sits at (a h, b h), h = 2^-k; every edge
    has length h and conductance 1/h (gamma = 1), as in the grid network of
    Section 6.2.
    """
    n = 2 ** k + 1
    h = 1.0 / (n - 1)
    ids = np.arange(n * n)
    ax, bx = ids % n, ids // n
    coords = np.stack([ax * h, bx * h], axis=1)
    hx = ids[ax < n - 1]
    vy = ids[bx < n - 1]
    E = np.concatenate([np.stack([hx, hx + 1], 1), np.stack([vy, vy + n], 1)]).astype(np.int64)
    m = E.shape[0]
    dirs = np.zeros((m, 2))
    dirs[: hx.size, 0] = 1.0
    dirs[hx.size:, 1] = 1.0
    return Network(2, coords, E, np.full(m, FIBER, np.int8), np.full(m, 1.0 / h),
                   np.full(m, 1.0 / h), dirs, (1.0, 1.0))


def subdivide(net: Network, k: int) -> Network:
    """Split every edge into k equal pieces of conductance k*c (series-equivalent).

    The original nodes keep their ids 0..n-1; the new interior nodes follow.
    """
    if k == 1:
        return net
    n, m = net.n_nodes, net.n_edges
    X = net.coords
    i, j = net.edges[:, 0], net.edges[:, 1]
    frac = np.arange(1, k) / k
    newpts = X[i][:, None, :] + frac[None, :, None] * (X[j] - X[i])[:, None, :]
    new_ids = n + np.arange(m * (k - 1)).reshape(m, k - 1)
    chain = np.concatenate([i[:, None], new_ids, j[:, None]], axis=1)
    E = np.stack([chain[:, :-1].ravel(), chain[:, 1:].ravel()], axis=1)
    rep = lambda v: np.repeat(v, k, axis=0)
    return Network(net.dim, np.concatenate([X, newpts.reshape(-1, net.dim)]), E,
                   rep(net.kind), rep(net.cond) * k, rep(net.stiff) * k, rep(net.dirs),
                   net.domain)


# ----------------------------------------------------------------------------
# problems
# ----------------------------------------------------------------------------

X_FACES = face_bit(0, 0) | face_bit(0, 1)


def scalar_band_problem(net: Network, H: float, f=None, star_set=STAR_INTERIOR, name="") -> Problem:
    """u = 0 at nodes with x < 0.01, u = 1 at x > 0.99; f = 0 unless given."""
    x = net.coords[:, 0]
    lo = np.nonzero(x < 0.01)[0]
    hi = np.nonzero(x > 0.99)[0]
    dd = np.concatenate([lo, hi])
    dv = np.concatenate([np.zeros(lo.size), np.ones(hi.size)])
    o = np.argsort(dd, kind="stable")
    ff = np.zeros(net.n_nodes) if f is None else np.asarray(f, dtype=np.float64)
    return Problem(net, 1, "scalar", dd[o].astype(np.int64), dv[o], ff, H, (X_FACES,),
                   star_set, name)


def truss_band_problem(net: Network, H: float, ux: float = 0.01, star_set=STAR_INTERIOR,
                       name="") -> Problem:
    """3 dofs per node: clamp all components at x < 0.01; u_x = ux at x > 0.99."""
    assert net.dim == 3
    x = net.coords[:, 0]
    lo = np.nonzero(x < 0.01)[0]
    hi = np.nonzero(x > 0.99)[0]
    dd = np.concatenate([3 * lo, 3 * lo + 1, 3 * lo + 2, 3 * hi])
    dv = np.concatenate([np.zeros(3 * lo.size), np.full(hi.size, ux)])
    o = np.argsort(dd, kind="stable")
    faces = (X_FACES, face_bit(0, 0), face_bit(0, 0))
    return Problem(net, 3, "truss3", dd[o].astype(np.int64), dv[o], np.zeros(3 * net.n_nodes),
                   H, faces, star_set, name)


def grid_heat_problem(k: int, H: float, star_set=STAR_ALL, patch=PATCH_SUPPORT) -> Problem:
    """Heat problem of Section 6.2 on the (2^k+1)^2 grid: Gamma = boundary, f = M1.

    (M1)(x) = 1/2 sum_{y~x} |x - y| (eq. 2.1 applied to the constant 1).  Stars
    sit at every mesh node and hold the nodes where the node's basis function
    is nonzero (the grid's nodes lie on the mesh lines, where this matters).
    """
    net = grid_network_2d(k)
    X = net.coords
    on_b = np.nonzero(np.any((X <= 0.0) | (X >= 1.0), axis=1))[0]
    lengths = np.linalg.norm(X[net.edges[:, 1]] - X[net.edges[:, 0]], axis=1)
    f = np.zeros(net.n_nodes)
    np.add.at(f, net.edges[:, 0], 0.5 * lengths)
    np.add.at(f, net.edges[:, 1], 0.5 * lengths)
    allf = X_FACES | face_bit(1, 0) | face_bit(1, 1)
    return Problem(net, 1, "scalar", on_b.astype(np.int64), np.zeros(on_b.size), f, H, (allf,),
                   star_set, f"grid{k}", patch=patch)


def fiber_heat_network(seed: int, total_length: float = 1000.0, r: float = 0.05) -> Network:
    """The uniform 2D fibre network of Section 6.1: fibres of length r with midpoints
    uniform in [-r/2, 1 + r/2]^2 and uniform angles, drawn until their clipped length
    (the total edge length |1|_M^2) reaches total_length; a node at every crossing,
    nodes closer than r * 1e-4 along a fibre merged, and only the components that
    reach the boundary of the square kept (the rest cannot carry the Dirichlet data)."""
    return fiber_network_2d(0, r, seed, midpoint_pad=0.5 * r, keep="boundary", total_length=total_length)


def fiber_heat_problem(net: Network, H: float, gamma=None, name="") -> Problem:
    """The heat problem of Section 6.2 on a network: Gamma = the boundary of the unit
    square (u = 0 there), f = M1 (eq. 2.1: half the length of the edges at a node),
    conductance gamma_xy / |x - y| (Example 3.2) with gamma = 1 or the given per-edge
    weights; stars at every mesh node holding the nodes where the node's basis
    function is nonzero."""
    from dataclasses import replace
    if gamma is not None:
        net = replace(net, cond=net.cond * np.asarray(gamma, np.float64))
    X = net.coords
    on_b = np.nonzero(np.any((X <= 0.0) | (X >= 1.0), axis=1))[0]
    lengths = np.linalg.norm(X[net.edges[:, 1]] - X[net.edges[:, 0]], axis=1)
    f = np.zeros(net.n_nodes)
    np.add.at(f, net.edges[:, 0], 0.5 * lengths)
    np.add.at(f, net.edges[:, 1], 0.5 * lengths)
    allf = X_FACES | face_bit(1, 0) | face_bit(1, 1)
    return Problem(net, 1, "scalar", on_b.astype(np.int64), np.zeros(on_b.size), f, H, (allf,),
                   STAR_ALL, name, patch=PATCH_SUPPORT)


def beam_triples(net: Network) -> np.ndarray:
    """Node triples (x, y, z, along) of the bending form (eq. bend): every pair of distinct
    neighbours y < z of a node x, with along = 1 when x-y and x-z are edges of one fibre
    (y, x, z collinear) and 0 at a joint of two fibres; ascending (x, y, z)."""
    E = net.edges
    f = net.fiber if net.fiber is not None else np.full(net.n_edges, -1, np.int64)
    node = np.concatenate([E[:, 0], E[:, 1]])
    other = np.concatenate([E[:, 1], E[:, 0]])
    ff = np.concatenate([f, f])
    o = np.lexsort((other, node))
    node, other, ff = node[o], other[o], ff[o]
    starts = np.concatenate([[0], np.nonzero(node[1:] != node[:-1])[0] + 1, [node.size]])
    out = []
    for a0, a1 in zip(starts[:-1], starts[1:]):
        for i in range(a0, a1):
            for j in range(i + 1, a1):
                along = int(ff[i] >= 0 and ff[i] == ff[j])
                out.append((node[i], other[i], other[j], along))
    return np.array(out, dtype=np.int64).reshape(-1, 4)


def _anchored_fibres(net: Network, dirichlet_fn) -> Network:
    """Without the fibres held at fewer than two nodes (a node of a fibre holds it when
    it is a Dirichlet node or a joint with another kept fibre): the bending form does not
    couple the out-of-plane rotation of a fibre about a single joint, so such a fibre
    would leave K singular.  Repeated until every fibre left is held twice.  Then, on
    the graph of the edges between non-Dirichlet nodes, only the components joined to at
    least two distinct Dirichlet nodes are kept: the in-plane bending form is invariant
    under a rigid rotation about a node, so a component held at one Dirichlet node
    (a pin) turns freely about it."""
    f = net.fiber
    E = net.edges
    inc = np.unique(np.stack([np.concatenate([f, f]), np.concatenate([E[:, 0], E[:, 1]])], axis=1), axis=0)
    dmask = dirichlet_fn(net.coords)
    alive = np.ones(f.max() + 1, bool)
    while True:
        live = alive[inc[:, 0]]
        nf = np.bincount(inc[live, 1], minlength=net.n_nodes)
        anchor = dmask | (nf >= 2)
        held = np.bincount(inc[live, 0], weights=anchor[inc[live, 1]].astype(float), minlength=alive.size)
        drop = alive & (held < 2)
        if not drop.any():
            break
        alive &= ~drop
    keep_e = alive[f]
    E = E[keep_e]
    n = net.n_nodes
    dE = dmask[E]
    inner = ~dE[:, 0] & ~dE[:, 1]
    A = sp.coo_matrix((np.ones(int(inner.sum())), (E[inner, 0], E[inner, 1])), shape=(n, n))
    _, comp = connected_components(A, directed=False)
    pin = dE[:, 0] ^ dE[:, 1]  # edges from a component to a Dirichlet node
    free_end = np.where(dE[pin, 0], E[pin, 1], E[pin, 0])
    pins = np.unique(np.stack([comp[free_end], np.where(dE[pin, 0], E[pin, 0], E[pin, 1])], axis=1), axis=0)
    good = np.bincount(pins[:, 0], minlength=comp.max() + 1) >= 2
    keep_edge = np.zeros(E.shape[0], bool)
    keep_edge[inner] = good[comp[E[inner, 0]]]
    keep_edge[pin] = good[comp[free_end]]
    keep_n = np.zeros(n, bool)
    keep_n[E[keep_edge, 0]] = True
    keep_n[E[keep_edge, 1]] = True
    new_id = -np.ones(n, np.int64)
    new_id[keep_n] = np.arange(int(keep_n.sum()))
    sel = np.nonzero(keep_e)[0][keep_edge]
    return Network(net.dim, net.coords[keep_n], new_id[net.edges[sel]], net.kind[sel], net.cond[sel],
                   net.stiff[sel], net.dirs[sel], net.domain, net.fiber[sel])


BEAM_E = 210e9      # Young's modulus of the steel wires of Section 6.3 (Pa)
BEAM_RW = 2.5e-3    # their radius (m)


def beam_problem(net: Network, H: float, lateral: bool, strain: float | None = None, name="") -> Problem:
    """The structural problems of Section 6.3 on a 2D fibre network: 3 displacement
    components per node (two in the plane, one lateral), the tensile form (eq. tensile)
    with gamma_xy = A E and the bending form (eq. bend) of the wire (radius BEAM_RW,
    Young's modulus BEAM_E) on the node triples of beam_triples.  Gamma = the sides
    x_1 = 0 and x_1 = 1, g(x) = [s x_1, 0, 0] there.
    lateral False: the pure displacement problem (s = 0.2, in-plane only: the lateral
    component is held at zero everywhere); True: the lateral load problem (s = 0.1, the
    load M g' with g' = [0, 0, -1e3]).  Stars at every mesh node, support patches.
    Parallel edges (two fibres running between the same two merged joints) count once:
    x ~ y is a relation between nodes, and a pair of them would make a triple with
    y = z."""
    assert net.dim == 2
    net = _anchored_fibres(net, lambda X: (X[:, 0] <= 0.0) | (X[:, 0] >= 1.0))
    _, first = np.unique(np.sort(net.edges, axis=1), axis=0, return_index=True)
    if first.size < net.n_edges:
        k = np.sort(first)
        net = Network(net.dim, net.coords, net.edges[k], net.kind[k], net.cond[k], net.stiff[k], net.dirs[k],
                      net.domain, net.fiber[k])
    from dataclasses import replace
    A = np.pi * BEAM_RW ** 2
    net = replace(net, stiff=np.full(net.n_edges, A * BEAM_E))
    s = (0.1 if lateral else 0.2) if strain is None else strain
    X = net.coords
    side = np.nonzero((X[:, 0] <= 0.0) | (X[:, 0] >= 1.0))[0]
    dd = [3 * side, 3 * side + 1]
    dv = [s * X[side, 0], np.zeros(side.size)]
    if lateral:
        dd.append(3 * side + 2)
        dv.append(np.zeros(side.size))
    else:
        allz = np.arange(net.n_nodes)
        dd.append(3 * allz + 2)
        dv.append(np.zeros(allz.size))
    dd = np.concatenate(dd)
    dv = np.concatenate(dv)
    o = np.argsort(dd, kind="stable")
    f = np.zeros(3 * net.n_nodes)
    if lateral:  # M g': half the length of the edges at a node times g'
        lengths = np.linalg.norm(X[net.edges[:, 1]] - X[net.edges[:, 0]], axis=1)
        m = np.zeros(net.n_nodes)
        np.add.at(m, net.edges[:, 0], 0.5 * lengths)
        np.add.at(m, net.edges[:, 1], 0.5 * lengths)
        f[2::3] = -1e3 * m
    faces = (X_FACES, X_FACES, X_FACES if lateral else (X_FACES | face_bit(1, 0) | face_bit(1, 1)))
    return Problem(net, 3, "beam", dd[o].astype(np.int64), dv[o], f, H, faces, STAR_ALL,
                   name, meta={"triples": beam_triples(net), "r_w": BEAM_RW}, patch=PATCH_SUPPORT)


def heat_weights(net: Network, seed: int, lo: float = 0.1, hi: float = 1.0) -> np.ndarray:
    """Per-edge weights gamma_xy ~ U[lo, hi] (the weighted fibre network of Section 6.2)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=net.n_edges)


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

def config_seed(config: int, replicate: int = 0) -> int:
    return 1000 * config + replicate


def config1(replicate: int = 0) -> Problem:
    """2D diffusion: 1000 fibers of length 0.1, H = 1/8, interior stars."""
    net = fiber_network_2d(1000, 0.1, config_seed(1, replicate))
    return scalar_band_problem(net, 1.0 / 8, name="c1-2d-1000fib-H8")


def config2(replicate: int = 0, n_fibers: int = 40000, H: float = 1.0 / 16) -> Problem:
    """3D diffusion: 40000 fibers of length 0.1, contacts below 0.004, H = 1/16."""
    net = fiber_network_3d(n_fibers, 0.1, 0.004, config_seed(2, replicate))
    return scalar_band_problem(net, H, name=f"c2-3d-{n_fibers}fib-H{round(1/H)}")


def config3(replicate: int = 0, n_fibers: int = 20000, H: float = 1.0 / 12) -> Problem:
    """3D structural (3 dofs per node) on the 3D generator, H = 1/12."""
    net = fiber_network_3d(n_fibers, 0.1, 0.004, config_seed(3, replicate), keep="clamped_x")
    return truss_band_problem(net, H, name=f"c3-truss-{n_fibers}fib-H{round(1/H)}")


def request_problem(seed: int, max_fibers: int = 20000, min_fibers: int = 500,
                    nodes_per_element: float = 300.0):
    """One request of the serving stream: network, H and 1..16 right-hand sides.

    The generator is 2D or 3D with probability 1/2, the fiber count
    log-uniform in [min_fibers, max_fibers], H chosen so that about
    ``nodes_per_element`` nodes fall in each coarse element, f uniform in
    [0, 1] at free nodes, Dirichlet data as in the 2D workload.
    Returns (problem, F) with F of shape (nrhs, n_nodes).
    """
    rng = np.random.default_rng(seed)
    is3d = rng.random() < 0.5
    nfib = int(round(np.exp(rng.uniform(np.log(min_fibers), np.log(max_fibers)))))
    nrhs = int(rng.integers(1, 17))
    if is3d:
        net = fiber_network_3d(nfib, 0.1, 0.004, seed + 7)
    else:
        net = fiber_network_2d(nfib, 0.1, seed + 7)
    d = net.dim
    nH = max(2, int(round((net.n_nodes / nodes_per_element) ** (1.0 / d))))
    F = rng.uniform(0.0, 1.0, size=(nrhs, net.n_nodes))
    prob = scalar_band_problem(net, 1.0 / nH, f=F[0], name=f"req{seed}-{d}d-{nfib}fib-nH{nH}")
    return prob, F
