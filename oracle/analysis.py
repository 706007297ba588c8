"""Network analysis of Section 6.1 (oracle; test infrastructure): the homogeneity and the
connectivity constants of the network assumptions, written out from their definitions.

Section 3.2 (network assumptions): for boxes B_R(x) of side 2R (half-open, with the upper
face included where it lies on the boundary of Omega),
    homogeneity   rho <= (2R)^-d |1|^2_{M,B_R(x)} <= sigma rho,
    connectivity  a connected subgraph G' of G that holds every edge with an endpoint in
                  B_R(x) and only edges with both endpoints in B_{R+R0}(x).
Section 2.2: (M_x v, v) = 1/2 sum_{y~x} |x - y| v(x)^2, so |1|^2_{M,w} = sum over the nodes
x in w of m_x = 1/2 sum_{y~x} |x - y|; (L_x v, v) = 1/2 sum_{y~x} (v(x) - v(y))^2 / |x - y|,
so L is the graph Laplacian with conductance 1/|x - y| per edge.
Lemma 3.5 (proof, Neumann case): lambda_2 of L' u = lambda M' u on G' (L', M' defined for
G' as L, M for G) gives mu(x, R) = R^-1 lambda_2^-1/2; mu = max over the boxes.

Section 6.1 evaluates both on the elements of regular grids with R^-1 = 4, 8, 16, 32, 64
and R0^-1 = 64, the subgraph with the fewest edges a breadth-first search finds.  Readings
(listed with their reasons in the design notes): the boxes are the cells of the grid of
side 2R over the unit square (R^-1 / 2 cells per axis); sigma is the largest box value over
the smallest (rho the smallest); the subgraph starts from the edges with an endpoint in the
box and joins its components one at a time, by the shortest path (in edges) that a
breadth-first search from the component holding the most nodes finds through edges with both
endpoints in B_{R+R0}; a box whose pieces cannot be joined that way has no subgraph.
"""
from __future__ import annotations

from collections import deque

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.sparse.csgraph import connected_components


def largest_component(net):
    """The network restricted to its largest connected component (Assumption 3.2 takes the
    network connected; Section 6.1 removes the pieces left disconnected along the boundary)."""
    from dataclasses import replace
    n = net.n_nodes
    E = net.edges
    A = sp.coo_matrix((np.ones(E.shape[0]), (E[:, 0], E[:, 1])), shape=(n, n))
    _, comp = connected_components(A, directed=False)
    used = np.zeros(n, dtype=bool)
    used[E.ravel()] = True
    big = int(np.argmax(np.bincount(comp[used])))
    keep_n = comp == big
    new_id = -np.ones(n, dtype=np.int64)
    new_id[keep_n] = np.arange(int(keep_n.sum()))
    ke = keep_n[E[:, 0]]
    fields = dict(coords=net.coords[keep_n], edges=new_id[E[ke]])
    for name in ("kind", "cond", "stiff", "dirs", "fiber"):
        v = getattr(net, name, None)
        if v is not None:
            fields[name] = v[ke]
    return replace(net, **fields)


def edge_lengths(net):
    X = net.coords
    return np.linalg.norm(X[net.edges[:, 1]] - X[net.edges[:, 0]], axis=1)


def node_mass(net):
    """m_x = 1/2 sum_{y~x} |x - y| (the diagonal of M)."""
    L = edge_lengths(net)
    m = np.zeros(net.n_nodes)
    np.add.at(m, net.edges[:, 0], 0.5 * L)
    np.add.at(m, net.edges[:, 1], 0.5 * L)
    return m


def box_index(coords, lo, hi, nb):
    """Cell of every node in the grid of nb cells per axis over [lo, hi]: half-open cells,
    the upper face included on the boundary of the domain.  Nodes outside get -1."""
    coords = np.asarray(coords, dtype=np.float64)
    d = coords.shape[1]
    idx = np.zeros(coords.shape[0], dtype=np.int64)
    ok = np.ones(coords.shape[0], dtype=bool)
    stride = 1
    for a in range(d):
        s = (coords[:, a] - lo[a]) * nb / (hi[a] - lo[a])
        e = np.minimum(np.floor(s), nb - 1).astype(np.int64)
        ok &= (s >= 0) & (coords[:, a] <= hi[a])
        idx += e * stride
        stride *= nb
    idx[~ok] = -1
    return idx


def in_box(coords, lo, hi, domain_hi):
    """Membership of B = prod [lo_i, hi_i) (closed above where hi_i is the domain's edge)."""
    coords = np.asarray(coords, dtype=np.float64)
    ok = np.ones(coords.shape[0], dtype=bool)
    for a in range(coords.shape[1]):
        top = coords[:, a] <= hi[a] if hi[a] >= domain_hi[a] else coords[:, a] < hi[a]
        ok &= (coords[:, a] >= lo[a]) & top
    return ok


def homogeneity(net, Rinv):
    """(2R)^-d |1|^2_{M,B} for every cell B of side 2R = 2 / Rinv, and (sigma, rho)."""
    d = net.dim
    nb = max(1, int(round(Rinv / 2)))
    side = 1.0 / nb
    m = node_mass(net)
    lo = np.zeros(d)
    hi = np.asarray(net.domain, dtype=np.float64)
    b = box_index(net.coords, lo, hi, nb)
    vals = np.bincount(b[b >= 0], weights=m[b >= 0], minlength=nb ** d) / side ** d
    rho = float(vals.min())
    return vals, (float(vals.max()) / rho if rho > 0 else np.inf), rho


def _components(Es):
    """Connected components of the graph of the edges Es: (nodes, component of each node)."""
    nodes, inv = np.unique(Es, return_inverse=True)
    inv = inv.reshape(Es.shape)
    k = nodes.size
    A = sp.coo_matrix((np.ones(Es.shape[0]), (inv[:, 0], inv[:, 1])), shape=(k, k))
    _, comp = connected_components(A, directed=False)
    return nodes, comp


def connecting_subgraph(net, lo, hi, R0):
    """Edge ids of the subgraph G' for the box B = [lo, hi) (reading in the module header),
    or None when its pieces cannot be joined inside B_{R+R0}."""
    X = net.coords
    E = net.edges
    dom = np.asarray(net.domain, dtype=np.float64)
    inside = in_box(X, lo, hi, dom)
    big = in_box(X, np.asarray(lo) - R0, np.asarray(hi) + R0, dom)
    chosen = inside[E[:, 0]] | inside[E[:, 1]]
    if not chosen.any():
        return np.zeros(0, dtype=np.int64)
    nbr = {}
    edge_of = {}
    for k in np.nonzero(big[E[:, 0]] & big[E[:, 1]])[0]:
        a, b = int(E[k, 0]), int(E[k, 1])
        key = (min(a, b), max(a, b))
        if key in edge_of:
            continue
        edge_of[key] = int(k)
        nbr.setdefault(a, []).append(b)
        nbr.setdefault(b, []).append(a)
    sel = set(np.nonzero(chosen)[0].tolist())
    while True:
        idx = np.array(sorted(sel))
        nodes, comp = _components(E[idx])
        if comp.max() == 0:
            return idx
        main = set(nodes[comp == int(np.argmax(np.bincount(comp)))].tolist())
        others = set(nodes.tolist()) - main
        # breadth-first from the main component through allowed edges to the nearest other piece
        prev = {u: None for u in main}
        q = deque(sorted(main))
        hit = None
        while q and hit is None:
            u = q.popleft()
            for v in sorted(nbr.get(u, ())):
                if v in prev:
                    continue
                prev[v] = u
                if v in others:
                    hit = v
                    break
                q.append(v)
        if hit is None:
            return None
        v = hit
        while prev[v] is not None:
            u = prev[v]
            sel.add(edge_of[(min(u, v), max(u, v))])
            v = u


def lambda2(net, edge_ids):
    """Second eigenvalue of L' u = lambda M' u on the subgraph of the given edges (L' with
    conductance 1/|x - y|, M' the half edge lengths at each node)."""
    E = net.edges[edge_ids]
    nodes, inv = np.unique(E, return_inverse=True)
    inv = inv.reshape(E.shape)
    n = nodes.size
    L = edge_lengths(net)[edge_ids]
    c = 1.0 / L
    i, j = inv[:, 0], inv[:, 1]
    Lm = sp.coo_matrix((np.concatenate([c, c, -c, -c]), (np.concatenate([i, j, i, j]),
                                                        np.concatenate([i, j, j, i]))), shape=(n, n)).tocsr()
    m = np.zeros(n)
    np.add.at(m, i, 0.5 * L)
    np.add.at(m, j, 0.5 * L)
    if n <= 1500:
        ev = sla.eigh(Lm.toarray(), np.diag(m), eigvals_only=True, subset_by_index=[0, 1])
        return float(ev[1])
    # shift-and-invert about a small negative shift: the two eigenvalues nearest it are 0, lambda_2
    shift = -1e-6 * float((Lm.diagonal() / m).min())
    ev = spla.eigsh(Lm, k=2, M=sp.diags(m), sigma=shift, which="LM", return_eigenvectors=False)
    return float(np.sort(ev)[1])


def connectivity(net, Rinv, R0, limit=None):
    """mu(x, R) = R^-1 lambda_2^-1/2 for every cell of side 2R = 2 / Rinv, and mu = their
    maximum, on the largest connected component of the network (cells without a subgraph are
    skipped and counted)."""
    net = largest_component(net)
    d = net.dim
    nb = max(1, int(round(Rinv / 2)))
    side = 1.0 / nb
    R = 1.0 / Rinv
    vals, skipped = [], 0
    cells = list(np.ndindex(*([nb] * d)))
    for c in cells[:limit]:
        lo = np.array(c, dtype=np.float64) * side
        ids = connecting_subgraph(net, lo, lo + side, R0)
        if ids is None or ids.size == 0:
            skipped += 1
            continue
        lam = lambda2(net, ids)
        vals.append(1.0 / (R * np.sqrt(lam)))
    vals = np.array(vals)
    return vals, (float(vals.max()) if vals.size else np.nan), skipped
