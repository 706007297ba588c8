"""Operator assembly and the Dirichlet lifting (oracle; test infrastructure).

Scalar model, Example 3.2 eq. (scalarmodel): (K_x v, v) = 1/2 sum_{y~x}
gamma_xy (v(x) - v(y))^2 / |x - y|.  Written per edge e = {i, j} with the
conductance c_e = gamma_xy / |x - y|, the bilinear form is
sum_e c_e (v_i - v_j)(w_i - w_j), i.e. K = sum_e c_e (d_i - d_j)(d_i - d_j)^T.

Structural model, eq. (tensile) with the lateral regularisation of the 3-dof
workload: each edge contributes c_e (v_i - v_j)^T (n n^T + 0.1 I)(w_i - w_j),
c_e = EA / L_eff.  Dofs are node-major (3*node + component).

Beam model (Example 3.3 with d = 2, n = 3; Section 6.3): K = K^(T) + K^(B).
eq. (tensile) without the lateral term: each edge adds gamma_xy / L (d . (v_i - v_j))^2,
d the unit edge direction, gamma_xy = A E.  eq. (bend): node x with neighbours y != z
adds, for k = 1, 2, gamma_xyz (L_y + L_z) / 2 (a_y + a_z)^2 per ordered pair (y, z),
a_w = (v(w) - v(x)) . eta^(w,k) / L_w, gamma_xyz = E I (L_y + L_z)^-2,
E I = gamma_xy r_w^2 / 4.  Readings: k = 2 (in the plane) with eta^(y,2) = d_xy x e_3 and
eta^(z,2) = -d_xz x e_3, the change of the angle between the two edges, so that the term
vanishes on rigid motions and a kink of a straight wire costs energy (with both normals
d_xw x e_3 as printed, a kink would cost nothing and a rigid rotation would); k = 1 (out
of the plane) as printed, eta^(1) = e_3 on both sides, for every pair (for an angled
pair no out-of-plane form of this kind vanishes on rotations about in-plane axes; the
Dirichlet sides remove those).  Each unordered pair appears twice in the ordered sum, so
it adds E I / (L_y + L_z) (a_y + a_z)^2 for each k.

Section 3: with u_hat = u + g, g the Dirichlet data extended by zero, the free
block solves A u_I = b with A = K_II and b = f_I - K_ID g_D.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def assemble(problem) -> sp.csr_matrix:
    """K on all n_nodes * ndof dofs as a CSR matrix (duplicates summed)."""
    net = problem.net
    n = net.n_nodes
    i = net.edges[:, 0]
    j = net.edges[:, 1]
    if problem.model == "scalar":
        c = net.cond
        rows = np.concatenate([i, j, i, j])
        cols = np.concatenate([i, j, j, i])
        vals = np.concatenate([c, c, -c, -c])
        K = sp.coo_matrix((vals, (rows, cols)), shape=(n, n))
        return K.tocsr()
    if problem.model == "truss3":
        c = net.stiff
        nv = net.dirs
        # 3x3 block of one edge: c (n n^T + 0.1 I)
        blk = c[:, None, None] * (nv[:, :, None] * nv[:, None, :] + 0.1 * np.eye(3)[None])
        R, C, V = [], [], []
        for a in range(3):
            for b in range(3):
                v = blk[:, a, b]
                R += [3 * i + a, 3 * j + a, 3 * i + a, 3 * j + a]
                C += [3 * i + b, 3 * j + b, 3 * j + b, 3 * i + b]
                V += [v, v, -v, -v]
        K = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))),
                          shape=(3 * n, 3 * n))
        return K.tocsr()
    if problem.model == "beam":
        c = net.stiff
        X = net.coords
        L = np.linalg.norm(X[j] - X[i], axis=1)
        d3 = np.zeros((net.n_edges, 3))
        d3[:, :2] = (X[j] - X[i]) / L[:, None]
        R, C, V = [], [], []
        for a in range(3):  # tensile: (c / L) b b^T, b = [d, -d]
            for b in range(3):
                v = c / L * d3[:, a] * d3[:, b]
                R += [3 * i + a, 3 * j + a, 3 * i + a, 3 * j + a]
                C += [3 * i + b, 3 * j + b, 3 * j + b, 3 * i + b]
                V += [v, v, -v, -v]
        T = problem.meta["triples"]
        x, y, z = T[:, 0], T[:, 1], T[:, 2]
        Ly = np.linalg.norm(X[y] - X[x], axis=1)
        Lz = np.linalg.norm(X[z] - X[x], axis=1)
        EI = c[0] * problem.meta["r_w"] ** 2 / 4.0  # gamma_xy = A E is the same on every edge
        cb = EI / (Ly + Lz)
        ty = (X[y] - X[x]) / Ly[:, None]
        tz = (X[z] - X[x]) / Lz[:, None]
        zero = np.zeros(T.shape[0])
        e3 = np.stack([zero, zero, zero + 1.0], axis=1)
        # k = 2: eta^(y) = d_xy x e_3, eta^(z) = -d_xz x e_3; k = 1: e_3 on both sides
        terms = [(np.stack([ty[:, 1], -ty[:, 0], zero], axis=1), np.stack([-tz[:, 1], tz[:, 0], zero], axis=1),
                  np.ones(T.shape[0])),
                 (e3, e3, np.ones(T.shape[0]))]
        nodes = [x, y, z]
        for ey, ez, on in terms:  # (cb on) g g^T, g over the 9 dofs of (x, y, z)
            gv = [-(ey / Ly[:, None] + ez / Lz[:, None]), ey / Ly[:, None], ez / Lz[:, None]]
            for p_ in range(3):
                for q_ in range(3):
                    for a in range(3):
                        for b in range(3):
                            R.append(3 * nodes[p_] + a)
                            C.append(3 * nodes[q_] + b)
                            V.append(cb * on * gv[p_][:, a] * gv[q_][:, b])
        K = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))),
                          shape=(3 * n, 3 * n))
        return K.tocsr()
    raise ValueError(problem.model)


def split(problem, K=None):
    """Free/Dirichlet split (Section 3).

    Returns (free, A, K_ID) with ``free`` the ascending free dofs, A = K_II and
    K_ID the free-by-Dirichlet block (columns in the order of
    problem.dirichlet_dofs).
    """
    if K is None:
        K = assemble(problem)
    ndof_total = K.shape[0]
    is_d = np.zeros(ndof_total, bool)
    is_d[problem.dirichlet_dofs] = True
    free = np.nonzero(~is_d)[0]
    K = K.tocsr()
    A = K[free][:, free].tocsr()
    KID = K[free][:, problem.dirichlet_dofs].tocsr()
    return free, A, KID


def lifted_rhs(problem, f, g, free, KID):
    """b = f_I - K_ID g_D (the right-hand side of the lifted problem, Section 3)."""
    return np.asarray(f, dtype=np.float64)[free] - KID @ np.asarray(g, dtype=np.float64)


def expand(problem, free, u_free, g):
    """u_hat on all dofs: u on free dofs, g on Dirichlet dofs."""
    out = np.zeros(problem.n_dof)
    out[free] = u_free
    out[problem.dirichlet_dofs] = g
    return out
