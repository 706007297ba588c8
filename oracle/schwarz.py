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
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .coarse import CoarseSpace, mesh_multi, mesh_shape


def star_mesh_nodes(nH, star_set):
    """Mesh nodes carrying a star, ascending: all of them, or the interior ones."""
    n_mesh = int(np.prod([n + 1 for n in nH]))
    out = []
    for k in range(n_mesh):
        m = mesh_multi(k, nH)
        if star_set == "all" or all(0 < m[i] < nH[i] for i in range(len(nH))):
            out.append(k)
    return out


def star_dofs(elem, k_multi, nH, W=None):
    """Free dofs whose host element touches mesh node k (the patch U(y_k)).

    With the Q1 values W (n, 2^d) given, only the dofs where phi_k is nonzero
    are kept ("support" patches): phi_k at a dof is W at the corner of the
    dof's host element that sits at y_k.
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
        for k in star_mesh_nodes(self.nH, star_set):
            S = star_dofs(elem, mesh_multi(k, self.nH), self.nH, Wsup)
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
        self.c0 = sla.cho_factor(self.coarse.A0, lower=True) if self.coarse.m0 else None

    # pieces of B, exposed so that each step can be checked on its own
    def coarse_term(self, r):
        """R_0^T A_0^{-1} R_0 r."""
        if self.c0 is None:
            return np.zeros_like(r)
        return self.coarse.prolong(sla.cho_solve(self.c0, self.coarse.restrict(r)))

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
