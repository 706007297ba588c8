"""CPU FP64 oracle for the two-level additive Schwarz PCG of Goertz, Hellman and
Malqvist, "Iterative solution of spatial network models by subspace
decomposition".

This package is TEST INFRASTRUCTURE.  Only the test-suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
The CUDA library never calls into it and shares no code with it: the oracle
assembles the operator, builds the coarse space and the stars, factors every
local and coarse matrix densely and runs textbook PCG, all in plain numpy /
scipy FP64, step by step in the paper's order.

Modules
-------
operator  assembly of K from an edge list (eqs. 2.2, scalarmodel, tensile), the
          beam model with the bending term (Example 3.3, eq. bend), the Dirichlet
          lifting of Section 3
coarse    half-open host elements and Q1 values (Section 2.3), the P1 space on
          the Kuhn simplices of the box mesh with the lowest-element rule
          (Remark 2.1), coarse dofs, the restriction R_0 and the Galerkin
          matrix A_0 (Section 4.1)
schwarz   star spaces V_j = V(U(y_j)), exact local solves and the additive
          preconditioner B = sum_j P_j K^{-1}-form (Section 4.1, eq. defPj)
pcg       preconditioned conjugate gradients (Section 4.2), flexible variant,
          convergence rates tau_l (Section 6.2)
solve     end-to-end solve of a problem
analysis  the homogeneity sigma and the connectivity constant mu of the network
          assumptions (Section 3.2, Lemma 3.5), as Section 6.1 evaluates them

Readings of the paper that the oracle fixes (each is listed with its reason
in the design notes of the repository):

* Q1 is the multilinear (tensor-product) space: 2^d basis values per element.
* tau_l is |e_l|_K / |e_{l-1}|_K (the printed ratio is inverted).
* Stars sit at interior mesh nodes ("interior") or at every mesh node ("all");
  a star at a boundary mesh node holds only the elements that exist.
* Coarse basis functions are truncated to free dofs; mesh nodes on a Dirichlet
  face of a component, and mesh nodes whose truncated basis function vanishes,
  carry no coarse dof.
* PCG stops on the recursive residual |r|_2 <= rtol |b|_2 and then checks the
  recomputed residual, restarting at most twice.
* Star membership: "element" patches (every node of the elements around y_j;
  for P1 the simplices with y_j as a vertex) or "support" patches (the nodes
  where phi_j is nonzero).
* A coarse function in the span of earlier ones (a pivot at most 1e-8 of its
  diagonal entry in natural-order elimination) is left out of A_0^{-1}.
* The beam model: every neighbour pair at a node, the in-plane term measuring
  the change of the angle between the two edges, the out-of-plane term as
  printed, E I / (L_y + L_z) per unordered pair and term.

Parity is pinned for every function by the not-gpu tests (closed forms,
invariants, a direct solve, the paper's grid experiment, hand-computed beam
energies, brute-force simplex location and the textbook P1 stiffness stencil);
none is unpinned.
"""
