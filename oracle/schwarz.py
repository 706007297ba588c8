"""Two-level additive Schwarz preconditioner (oracle; test infrastructure).

Section 4.1: V_0 = V_H and V_j = V(U(y_j)), the functions that vanish outside
the patch of elements whose closure contains mesh node y_j.  P_j is the
K-orthogonal projection onto V_j (eq. defPj); for a subspace spanned by the
columns of E_j (unit vectors of the star's free dofs) it is
P_j = E_j A_j^{-1} E_j^T A with A_j = E_j^T A E_j, and for V_0
P_0 = R_0^T A_0^{-1} R_0 A.  Section 4.2 applies PCG to P = sum_j P_j = B A
with

    B r = R_0^T A_0^{-1} R_0 r + sum_j E_j A_j^{-1} E_j^T r.

Which nodes a star holds (the problem's ``patch``):

* "element": U(y_j) is the union of the half-open elements whose closure
  contains y_j (Section 2.3), so a node belongs to it iff its host element is
  one of the elements around y_j.  This is the star of the workloads ("the
  2^d-element patch around a mesh node"); with stars at interior mesh nodes
  only it is the reading that still covers the nodes on the Neumann faces.
* "support": only the nodes where phi_j is nonzero, i.e. those at max-norm
  distance below H from y_j.  The proof of Lemma 4.1 places its local parts
  (v - I v) phi_j in V_j, and these vanish wherever phi_j does, so this is the
  smallest star the stable decomposition needs.  It differs from "element"
  only at nodes on the outer boundary of the patch, which the paper's grid
  network (Section 6.2) has in number; with it the grid's rates agree with
  Table lap_conv.

Every A_j and A_0 is factored densely by Cholesky; the local terms are added
in ascending star order.

A rank-deficient coarse basis.  V_0 = V_H is the span of the basis functions
truncated to the free dofs, and these can be linearly dependent (a function
whose support holds few free nodes may be a combination of its neighbours
there); A_0 = R_0 A R_0^T is then singular, but the projection P_0 onto the
span is still defined.  The oracle keeps a basis of the span: Cholesky of A_0
in the coarse-dof order, where a function whose pivot (its part A-orthogonal
to the functions kept before it) is at most COARSE_DROP = 1e-8 times its
diagonal entry lies in their span and is left out.  Exactly dependent
functions leave pivots at rounding level (3e-11 and below on the sparse
networks here), independent ones 1e-6 and above; 1e-8 sits between, on a
logarithmic scale.  With K the kept functions,
P_0 = R_K^T A_KK^{-1} R_K A, which equals R_0^T A_0^+ R_0 A.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .coarse import CoarseSpace, mesh_multi, mesh_shape


COARSE_DROP = 1e-8  # relative pivot at or below which a coarse function is in the span of earlier ones


def coarse_basis(A0, tol=COARSE_DROP):
    """Kept coarse dofs and the Cholesky factor of A_0 on them.

    Cholesky in the coarse-dof order; dof k is left out when its pivot
    d_k = A0[k,k] - sum over kept j < k of L[k,j]^2 is at most tol * A0[k,k].
    When no pivot is that small this is LAPACK's Cholesky of A_0 (the same
    pivots); otherwise the elimination is written out with the drops.
    """
    m = A0.shape[0]
    diag = np.diag(A0).copy()
    try:
        L = np.linalg.cholesky(A0)
        if np.all(np.diag(L) ** 2 > tol * diag):
            return np.arange(m), (L, True)
    except np.linalg.LinAlgError:
        pass
    S = A0.copy()                      # the Schur complement of the kept dofs so far
    keep = np.zeros(m, dtype=bool)
    for k in range(m):
        d = S[k, k]
        if not d > tol * diag[k]:
            continue
        keep[k] = True
        col = S[k + 1:, k] / d
        S[k + 1:, k + 1:] -= np.outer(col, S[k, k + 1:])
    K = np.nonzero(keep)[0]
    return K, (np.linalg.cholesky(A0[np.ix_(K, K)]), True)


def star_mesh_nodes(nH, star_set):
    """Mesh nodes carrying a star, ascending: all of them, or the interior ones."""
    n_mesh = int(np.prod([n + 1 for n in nH]))
    out = []
    for k in range(n_mesh):
        m = mesh_multi(k, nH)
        if star_set == "all" or all(0 < m[i] < nH[i] for i in range(len(nH))):
            out.append(k)
    return out


def star_dofs(elem, k_multi, nH, W=None, V=None):
    """Free dofs whose host element touches mesh node k (the patch U(y_k)).

    With the basis values W (n, 2^d) given, only the dofs where phi_k is nonzero
    are kept ("support" patches): phi_k at a dof is W at the corner of the
    dof's host element that sits at y_k.  With the P1 vertex mask V (n, 2^d)
    given (Remark 2.1, element patches), only the dofs whose host simplex has
    y_k as a vertex are kept.
    """
    inside = np.ones(elem.shape[0], dtype=bool)
    for i in range(len(nH)):
        inside &= (elem[:, i] == k_multi[i] - 1) | (elem[:, i] == k_multi[i])
    S = np.nonzero(inside)[0]
    if W is not None and S.size:
        corner = np.zeros(S.size, dtype=np.int64)
        for i in range(len(nH)):
            corner += (k_multi[i] - elem[S, i]) << i
        S = S[W[S, corner] != 0.0]
    if V is not None and S.size:
        corner = np.zeros(S.size, dtype=np.int64)
        for i in range(len(nH)):
            corner += (k_multi[i] - elem[S, i]) << i
        S = S[V[S, corner]]
    return S


class SchwarzPreconditioner:
    """B of Section 4.2 for the free-dof matrix A of a problem.

    ``local`` chooses the exact local solver: "dense" (dense Cholesky of every
    A_j, the default) or "sparse" (a sparse LU factorisation, for patches too
    large to hold densely).
    """

    def __init__(self, problem, free, A, local: str = "dense", star_set: str | None = None):
        self.A = A.tocsr()
        self.coarse = CoarseSpace(problem, free, self.A)
        self.nH = mesh_shape(problem)
        star_set = problem.star_set if star_set is None else star_set
        self.star_mesh = []
        self.stars = []
        self.factors = []
        self.local = local
        elem = self.coarse.elem
        self.patch = getattr(problem, "patch", "element")
        Wsup = self.coarse.W if self.patch == "support" else None
        Vel = self.coarse.V if self.patch != "support" else None  # P1 element patches
        for k in star_mesh_nodes(self.nH, star_set):
            S = star_dofs(elem, mesh_multi(k, self.nH), self.nH, Wsup, Vel)
            if S.size == 0:
                continue
            Aj = self.A[S][:, S]
            if local == "dense":
                fac = sla.cho_factor(Aj.toarray(), lower=True)
            else:
                fac = spla.splu(Aj.tocsc())
            self.star_mesh.append(k)
            self.stars.append(S)
            self.factors.append(fac)
        self.c0 = None
        self.coarse_kept = np.zeros(0, dtype=np.int64)
        if self.coarse.m0:
            self.coarse_kept, self.c0 = coarse_basis(self.coarse.A0)

    # pieces of B, exposed so that each step can be checked on its own
    def coarse_solve(self, rc):
        """z_c with z_K = A_KK^{-1} r_K on the kept coarse dofs, zero on the others."""
        zc = np.zeros_like(rc)
        if self.c0 is not None:
            K = self.coarse_kept
            zc[K] = sla.cho_solve(self.c0, rc[K])
        return zc

    def coarse_term(self, r):
        """R_0^T A_0^{-1} R_0 r (A_0^{-1} on the kept basis of V_H)."""
        if self.c0 is None:
            return np.zeros_like(r)
        return self.coarse.prolong(self.coarse_solve(self.coarse.restrict(r)))

    def local_solve(self, j, rj):
        if self.local == "dense":
            return sla.cho_solve(self.factors[j], rj)
        return self.factors[j].solve(rj)

    def star_term(self, r):
        """sum_j E_j A_j^{-1} E_j^T r, stars in ascending order."""
        z = np.zeros_like(r)
        for j, S in enumerate(self.stars):
            z[S] += self.local_solve(j, r[S])
        return z

    def apply(self, r):
        """z = B r."""
        z = self.coarse_term(r)
        for j, S in enumerate(self.stars):
            z[S] += self.local_solve(j, r[S])
        return z

    def dense_B(self):
        """B as a dense matrix (tiny problems only)."""
        n = self.A.shape[0]
        B = np.zeros((n, n))
        I = np.eye(n)
        for i in range(n):
            B[:, i] = self.apply(I[:, i])
        return B

    @property
    def n_stars(self):
        return len(self.stars)

    @property
    def star_sizes(self):
        return np.array([S.size for S in self.stars], dtype=np.int64)
