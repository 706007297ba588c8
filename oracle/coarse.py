"""Mesh, Q1 basis values on network nodes and the coarse space V_H (oracle).

Section 2.3: the mesh T_H of Omega = prod [0, l_i] has n_i = l_i / H elements
per axis.  Elements are half-open boxes B_{H/2}(x) = prod [x_i - H/2, x_i + H/2)
that also contain their upper face where it lies on the boundary of Omega,
so every point belongs to exactly one element; along axis i the host element
of a node at x_i is e_i = min(floor(x_i * n_i / l_i), n_i - 1).

Q1 (multilinear) basis: with xi_i = x_i n_i / l_i - e_i in [0, 1] and corner
c in {0,1}^d of the host element, phi_{e+c}(x) = prod_i (xi_i if c_i else
1 - xi_i).  Mesh nodes y_k are numbered lexicographically with axis 0 fastest:
k = sum_i k_i s_i, s_0 = 1, s_i = prod_{j<i} (n_j + 1).  Corners are numbered
c = sum_i c_i 2^i.

P1 on simplices (Remark 2.1), for the Kuhn triangulation of the same box mesh:
each box is split into the d! simplices S_pi = {t : t_pi(0) >= ... >= t_pi(d-1)}
(pi a permutation of the axes), with vertices at the box corners whose bit sets
are the prefixes {pi(0), .., pi(j-1)}, j = 0..d; the simplices are shape regular
and aligned with the box faces.  Elements are numbered box by box (boxes in the
linear order above), the d! simplices of a box by the lexicographic order of pi.
A node goes to the lowest-numbered element whose closure holds it: along each
axis the lowest box, e_i = min(max(ceil(x_i n_i / l_i) - 1, 0), n_i - 1) (a point
on an interior box face belongs to the box below), then the lexicographically
first pi along which t is non-increasing.  The basis function of a vertex is its
barycentric coordinate: lambda_0 = 1 - t_pi(0), lambda_j = t_pi(j-1) - t_pi(j),
lambda_d = t_pi(d-1); it is zero at the other corners of the box.

Coarse dofs (the basis of V_H, ordered m_0 first): the pair (mesh node k,
component a) is a coarse dof unless y_k lies on a Dirichlet face of
component a, or phi_k vanishes at every free dof of component a (its
truncation to the free dofs is the zero function).  R_0 has one row per
coarse dof, R_0[(k,a), (x,a)] = phi_k(x) at free dofs; A_0 = R_0 A R_0^T is
the Galerkin matrix of the coarse projection P_0 (Section 4.1, eq. defPj).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def mesh_shape(problem):
    return tuple(int(round(l / problem.H)) for l in problem.net.domain)


def host_elements(coords, domain, nH):
    """Element multi-index of every node by the half-open box rule."""
    coords = np.asarray(coords, dtype=np.float64)
    d = coords.shape[1]
    e = np.empty(coords.shape, dtype=np.int64)
    for i in range(d):
        e[:, i] = np.minimum(np.floor(coords[:, i] * nH[i] / domain[i]), nH[i] - 1).astype(np.int64)
    return e


def host_simplices(coords, domain, nH):
    """Remark 2.1 on the Kuhn triangulation: (box multi-index e (n, d), permutation
    index of the host simplex (n,), local coordinates t (n, d)) by the lowest-element
    rule; permutations are numbered in the lexicographic order of itertools."""
    coords = np.asarray(coords, dtype=np.float64)
    d = coords.shape[1]
    e = np.empty(coords.shape, dtype=np.int64)
    t = np.empty(coords.shape)
    for i in range(d):
        s = coords[:, i] * nH[i] / domain[i]
        e[:, i] = np.minimum(np.maximum(np.ceil(s) - 1, 0), nH[i] - 1).astype(np.int64)
        t[:, i] = s - e[:, i]
    perms = list(itertools.permutations(range(d)))
    index = {p: j for j, p in enumerate(perms)}
    order = np.argsort(-t, axis=1, kind="stable")   # t non-increasing, ties: smaller axis first
    pidx = np.array([index[tuple(int(a) for a in row)] for row in order], dtype=np.int64)
    return e, pidx, t


def p1_values(t, pidx, d):
    """Barycentric coordinates of every node in its host simplex, as values at the
    2^d corners of the host box (zero at the corners that are not vertices), and the
    mask of the corners that are vertices: arrays (n, 2^d)."""
    perms = list(itertools.permutations(range(d)))
    n = t.shape[0]
    W = np.zeros((n, 2 ** d))
    V = np.zeros((n, 2 ** d), dtype=bool)
    for r in range(n):
        p = perms[pidx[r]]
        c = 0
        prev = 1.0
        for j in range(d + 1):
            cur = t[r, p[j]] if j < d else 0.0
            W[r, c] = prev - cur
            V[r, c] = True
            if j < d:
                c |= 1 << p[j]
                prev = cur
    return W, V


def corner_list(d):
    """Corners c in {0,1}^d in the order c = sum_i c_i 2^i."""
    return [tuple((c >> i) & 1 for i in range(d)) for c in range(2 ** d)]


def q1_values(coords, domain, nH, e=None):
    """phi at the 2^d corners of each node's host element: array (n, 2^d)."""
    coords = np.asarray(coords, dtype=np.float64)
    d = coords.shape[1]
    if e is None:
        e = host_elements(coords, domain, nH)
    xi = np.empty(coords.shape)
    for i in range(d):
        xi[:, i] = coords[:, i] * nH[i] / domain[i] - e[:, i]
    W = np.ones((coords.shape[0], 2 ** d))
    for ci, c in enumerate(corner_list(d)):
        for i in range(d):
            W[:, ci] *= xi[:, i] if c[i] else (1.0 - xi[:, i])
    return W


def mesh_strides(nH):
    s = [1]
    for i in range(len(nH) - 1):
        s.append(s[-1] * (nH[i] + 1))
    return s


def mesh_index(multi, nH):
    s = mesh_strides(nH)
    return sum(int(multi[i]) * s[i] for i in range(len(nH)))


def mesh_multi(k, nH):
    out = []
    for i in range(len(nH)):
        out.append(k % (nH[i] + 1))
        k //= nH[i] + 1
    return tuple(out)


def on_faces(multi, nH, facemask):
    """True if mesh node multi-index lies on any face in the bitmask."""
    for a in range(len(nH)):
        if (facemask >> (2 * a)) & 1 and multi[a] == 0:
            return True
        if (facemask >> (2 * a + 1)) & 1 and multi[a] == nH[a]:
            return True
    return False


class CoarseSpace:
    """The restriction R_0 and the Galerkin matrix A_0 for a problem's free dofs."""

    def __init__(self, problem, free, A):
        net = problem.net
        d = net.dim
        nd = problem.ndof
        self.nH = mesh_shape(problem)
        nH = self.nH
        node_of = free // nd
        comp_of = free % nd
        X = net.coords[node_of]
        self.space = getattr(problem, "coarse", "q1")
        self.V = None  # P1: corners of the host box that are vertices of the host simplex
        if self.space == "p1":
            self.elem, self.simplex, t = host_simplices(X, net.domain, nH)
            self.W, self.V = p1_values(t, self.simplex, d)
        else:
            self.elem = host_elements(X, net.domain, nH)
            self.W = q1_values(X, net.domain, nH, self.elem)
        strides = mesh_strides(nH)
        corners = corner_list(d)
        n_mesh = int(np.prod([n + 1 for n in nH]))
        # mesh node index of every (free dof, corner)
        K = np.zeros((free.size, 2 ** d), dtype=np.int64)
        for ci, c in enumerate(corners):
            K[:, ci] = sum((self.elem[:, i] + c[i]) * strides[i] for i in range(d))
        self.mesh_of = K
        # candidate coarse dofs: (k, a) with a nonzero value at some free dof of component a
        support = np.zeros((n_mesh, nd), dtype=bool)
        nz = self.W != 0.0
        for ci in range(2 ** d):
            support[K[nz[:, ci], ci], comp_of[nz[:, ci]]] = True
        keep = np.zeros((n_mesh, nd), dtype=bool)
        for k in range(n_mesh):
            m = mesh_multi(k, nH)
            for a in range(nd):
                keep[k, a] = support[k, a] and not on_faces(m, nH, problem.gamma_faces[a])
        self.coarse_index = -np.ones((n_mesh, nd), dtype=np.int64)
        flat = np.nonzero(keep.ravel())[0]          # order: k ascending, component ascending
        self.coarse_index.ravel()[flat] = np.arange(flat.size)
        self.m0 = int(flat.size)
        rows, cols, vals = [], [], []
        for ci in range(2 ** d):
            ck = self.coarse_index[K[:, ci], comp_of]
            ok = ck >= 0
            rows.append(ck[ok])
            cols.append(np.nonzero(ok)[0])
            vals.append(self.W[ok, ci])
        self.R0 = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(self.m0, free.size)).tocsr()
        self.A0 = (self.R0 @ A @ self.R0.T).toarray()

    def restrict(self, r):
        """r_c = R_0 r."""
        return self.R0 @ r

    def prolong(self, zc):
        """R_0^T z_c."""
        return self.R0.T @ zc
