"""Operator assembly and the Dirichlet lifting (oracle; test infrastructure).

Scalar model, Example 3.2 eq. (scalarmodel): (K_x v, v) = 1/2 sum_{y~x}
gamma_xy (v(x) - v(y))^2 / |x - y|.  Written per edge e = {i, j} with the
conductance c_e = gamma_xy / |x - y|, the bilinear form is
sum_e c_e (v_i - v_j)(w_i - w_j), i.e. K = sum_e c_e (d_i - d_j)(d_i - d_j)^T.

Structural model, eq. (tensile) with the lateral regularisation of the 3-dof
workload: each edge contributes c_e (v_i - v_j)^T (n n^T + 0.1 I)(w_i - w_j),
c_e = EA / L_eff.  Dofs are node-major (3*node + component).

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
