/*
 * spnet.h -- C ABI of the GB300 solver for spatial network models.
 *
 * The library solves (K u, v) = (f, v) for u in V (the node functions that
 * vanish on the Dirichlet set, Section 3, eq. weakform) by preconditioned
 * conjugate gradients (Section 4.2) with the two-level additive Schwarz
 * preconditioner of Section 4.1:
 *
 *     B r = R_0^T A_0^{-1} R_0 r + sum_j E_j A_j^{-1} E_j^T r,
 *
 * where R_0 evaluates the Q1 basis of the Cartesian mesh T_H (Section 2.3) at
 * the network's free dofs, A_0 = R_0 A R_0^T, and A_j is the block of the free
 * matrix A on the patch U(y_j) of mesh node y_j (eq. defPj).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: SPNET_OK (0) or a negative SPNET_ERR_* code;
 *    spnet_last_error() gives the message of the last failure on the calling
 *    thread.
 *  - `mem` says where every array argument of that call lives:
 *    SPNET_MEM_HOST (ordinary host memory) or SPNET_MEM_DEVICE (device memory
 *    of the current CUDA device).  Input arrays are borrowed for the duration
 *    of the call and copied; output arrays are owned by the caller.
 *  - Dofs are numbered node-major: dof = ndof * node + component.
 *  - `stream` is a cudaStream_t (passed as void*); 0 means the legacy default
 *    stream.  All work of an operator and of its preconditioners is issued on
 *    the operator's stream.  Calls return after their results are complete.
 *  - Handles are opaque and owned by the library until *_destroy.  A
 *    preconditioner keeps a reference to its operator: destroy it first.
 *  - Nothing here is thread-safe per handle; distinct handles may be used
 *    from distinct threads.
 */
#ifndef SPNET_H
#define SPNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPNET_OK 0
#define SPNET_ERR_BAD_INPUT (-1)       /* malformed arguments, asymmetric K, NaN, bad indices */
#define SPNET_ERR_NOT_SPD (-2)         /* a pivot <= 0 in a local or coarse factorisation */
#define SPNET_ERR_NO_MEMORY (-3)       /* device allocation failed */
#define SPNET_ERR_NO_CONVERGENCE (-4)  /* maxit reached; the iterate is still returned */
#define SPNET_ERR_TIMEOUT (-5)         /* a bounded device wait expired (reserved: no call of
                                          this build waits on the device with a limit, so
                                          none returns it) */
#define SPNET_ERR_CUDA (-6)            /* a CUDA runtime error */
#define SPNET_ERR_UNSUPPORTED (-7)     /* a size beyond the limits of this build */
#define SPNET_ERR_BAD_H (-8)           /* l_i / H is not an integer >= 1 */
#define SPNET_ERR_CANCELLED (-9)       /* a served request was cancelled before admission */

#define SPNET_MEM_HOST 0
#define SPNET_MEM_DEVICE 1

#define SPNET_MODEL_SCALAR 0  /* eq. scalarmodel: K = sum_e c_e (d_i - d_j)(d_i - d_j)^T */
#define SPNET_MODEL_TRUSS3 1  /* eq. tensile + lateral term: 3x3 blocks c_e (n n^T + 0.1 I) */

#define SPNET_PREC_FP64 0   /* factors, coarse inverse and local solves in FP64 */
#define SPNET_PREC_MIXED 1  /* factors and coarse inverse stored and applied in FP32 */

#define SPNET_STARS_INTERIOR 0  /* stars at mesh nodes off the boundary of Omega */
#define SPNET_STARS_ALL 1       /* stars at every mesh node y_1..y_m (Section 4.1) */

/* Which free dofs the star of mesh node y_j holds (Sections 2.3, 4.1). */
#define SPNET_PATCH_ELEMENT 0  /* every dof whose host element touches y_j: Q1, the union of
                                  the (up to 2^d) boxes around y_j; P1, the simplices that have
                                  y_j as a vertex */
#define SPNET_PATCH_SUPPORT 1  /* only the dofs where the basis function of y_j is nonzero
                                  (Q1: max-norm distance below H): the space the local parts
                                  (v - I v) phi_j of the proof of Lemma 4.1 live in.  Differs
                                  from ELEMENT only at dofs on the outer boundary of the patch */

/* The coarse space V_H (Section 2.3, Remark 2.1). */
#define SPNET_COARSE_Q1 0  /* multilinear Lagrange functions on the box mesh; a node's host element
                              is the half-open box min(floor(x_i n_i / l_i), n_i - 1) */
#define SPNET_COARSE_P1 1  /* continuous piecewise affine functions on the Kuhn triangulation of
                              the box mesh (Remark 2.1): each box split into the d! simplices
                              {t_pi(0) >= ... >= t_pi(d-1)} (t the local coordinates, pi a
                              permutation of the axes); elements numbered box by box, the
                              simplices of a box by the lexicographic order of pi; a node goes
                              to the lowest-numbered element whose closure holds it.  The basis
                              values are the barycentric coordinates; ELEMENT patches hold the
                              dofs whose host simplex has y_j as a vertex */

typedef struct spnet_op_s* spnet_op_t;
typedef struct spnet_pc_s* spnet_pc_t;

typedef struct {
  int precision;     /* SPNET_PREC_* (default SPNET_PREC_MIXED) */
  int star_set;      /* SPNET_STARS_* (default SPNET_STARS_INTERIOR) */
  int flexible;      /* 1: Polak-Ribiere beta (r, z - z_old)/(r_old, z_old); 0: textbook
                        beta; -1: flexible iff precision is MIXED (default -1) */
  int max_restarts;  /* restarts from the recomputed residual (default 2) */
  int batch_rhs;     /* right-hand sides pcg_solve steps together: 0 or 1 one at a time
                        (default); 2..32 blocks of up to that many (fewer where the largest
                        star's solve vector for that many does not fit a block's shared
                        memory), each right-hand side with its own scalars and stop test;
                        the matrix, the star factors and the coarse tiles are read once
                        per block */
  int star_map;      /* warps per block of the one-vector star solve: 0 picks it per size
                        class (stars, largest star, entries per star) by timing the candidates
                        once per process (default); 1..8 fixes it.  Every warp solves whole
                        stars, so the choice changes no result */
  int patch;         /* SPNET_PATCH_* (default SPNET_PATCH_ELEMENT) */
  int no_panels;     /* 1: solve the dense block that ends a large star's elimination level by
                        level also in blocks of right-hand sides; 0 (default): in mixed
                        precision with batch_rhs >= 2, blocks of 32 nodes or more are solved
                        by 16-row panels with tensor-core products (TF32 inputs split in high
                        and low parts, FP32 accumulation) */
  int coarse_space;  /* SPNET_COARSE_* (default SPNET_COARSE_Q1) */
  int reserved[7];
} spnet_options;

typedef struct {
  int iterations;          /* products with A (CG steps) */
  int restarts;            /* restarts from the recomputed residual */
  int converged;           /* 1 if the recomputed relative residual <= rtol */
  int status;              /* SPNET_OK or SPNET_ERR_NO_CONVERGENCE */
  double relres;           /* ||b - A x||_2 / ||b||_2, recomputed in FP64 at the end */
  double relres_recursive; /* the recursive residual when the iteration stopped */
  double solve_ms;         /* device time of this right-hand side's solve */
  double reserved[4];
} spnet_stats;

typedef struct {
  int64_t n_dof, n_free, n_dirichlet, nnz_ff, nnz_fd;
  int dim, ndof;
  int64_t reserved[6];
} spnet_op_info;

typedef struct {
  int nH[3];            /* elements per axis */
  int n_elem, n_mesh;   /* elements, mesh nodes */
  int m0;               /* coarse dofs (dimension of V_H) */
  int n_stars;          /* non-empty stars */
  int max_star;         /* largest star (dofs) */
  int64_t sum_star;     /* sum of star sizes */
  int64_t factor_nnz;   /* off-diagonal entries of all local Cholesky factors */
  int64_t total_levels; /* sum over stars of the level count of the local solves */
  int max_levels;       /* largest level count of one star */
  int precision, star_set, flexible;
  double setup_ms;      /* device time of setup_preconditioner */
  int64_t device_bytes; /* device memory held by the preconditioner */
  int64_t star_stream_bytes; /* bytes one star solve reads from its solve streams
                                (headers, inverse permutations, entries) */
  int64_t star_warps_per_block; /* the star solve's mapping in use (see spnet_options.star_map) */
  int64_t coarse_dropped;       /* coarse functions left out of A_0^{-1} as linear combinations
                                   of earlier ones (see setup_preconditioner) */
  int64_t panel_stars;          /* stars whose dense block the k-right-hand-side solve runs by
                                   panels on tensor cores (see spnet_options.no_panels) */
  int64_t tuned;                /* the tuner's other choices: SpMV lanes per row
                                   + 256 * right-hand sides per warp of the batched star solve
                                   (0: chosen by the block width) */
} spnet_pc_info;

/* spnet_assemble -- assemble K on all n_nodes*ndof dofs from an edge list.
 *
 * Scalar model (model = SPNET_MODEL_SCALAR, ndof = 1), Example 3.2
 * eq. (scalarmodel): every edge e = {i, j} with conductance coef[e] =
 * gamma_e / |x_i - x_j| adds coef[e] (d_i - d_j)(d_i - d_j)^T.
 * Structural model (SPNET_MODEL_TRUSS3, ndof = 3), eq. (tensile) plus a
 * lateral term: the edge adds the 3x3 block coef[e] (n n^T + 0.1 I) with
 * n = dirs[3e..3e+2] (unit) in the pattern [[+,-],[-,+]].
 *
 * edges: [2*n_edges] int64 node ids (i, j), i != j; coef: [n_edges];
 * dirs: [3*n_edges] for TRUSS3, ignored (may be NULL) for SCALAR.
 * Output CSR (caller-owned, in `mem`): row_ptr [n_dof+1], col [cap_nnz],
 * val [cap_nnz]; columns sorted ascending within each row, parallel edges
 * summed, the diagonal always present.  cap_nnz >= ndof*ndof*(n_nodes +
 * 2*n_edges) always suffices.  *nnz_out (host) receives the entry count.
 * Errors: BAD_INPUT (bad ids, self-loops, non-finite coefficients), UNSUPPORTED
 * (cap_nnz too small or more than 2^31-1 entries).
 */
int spnet_assemble(int model, int64_t n_nodes, int64_t n_edges, const int64_t* edges,
                   const double* coef, const double* dirs, int mem, void* stream,
                   int64_t* row_ptr, int32_t* col, double* val, int64_t cap_nnz,
                   int64_t* nnz_out);

/* spnet_assemble_beam -- K of the structural model of Example 3.3 for a planar network
 * (d = 2, n = 3: two displacement components in the plane, one lateral), Section 6.3.
 *
 * K = K^(T) + K^(B) on 3 * n_nodes dofs (node-major).  eq. (tensile) without the lateral
 * term: each edge e = {i, j} of length L adds (coef[e] / L) (d . (v_i - v_j))^2, d the unit
 * edge direction (coef: gamma_xy = A E).  eq. (bend): each triple (x, y, z, along) of
 * triples [4 * n_triples] (x with two distinct neighbours y, z; the fourth entry is ignored
 * here) adds, for k = 1, 2, EI / (L_y + L_z) (a_y + a_z)^2 with a_w = (v(w) - v(x)) .
 * eta_w / L_w: k = 2 with eta_y = d_xy x e_3 and eta_z = -d_xz x e_3 (the change of the angle
 * between the two edges), k = 1 with eta_y = eta_z = e_3 (this is the paper's form summed over
 * ordered pairs, each unordered pair counted twice; the sign of eta_z for k = 2 is read so
 * that a kink costs energy and a rigid rotation in the plane does not).  EI = E I, the
 * wire's bending stiffness (gamma_xyz = EI (L_y + L_z)^-2).  coords [2 * n_nodes].
 * Output CSR as spnet_assemble (rows sorted; a node's rows couple it to itself, its edge
 * neighbours and the other members of its triples).  Errors: BAD_INPUT (bad ids, repeated
 * members of a triple, non-finite values), UNSUPPORTED (cap_nnz too small; a node coupled to
 * more than 64 nodes).
 */
int spnet_assemble_beam(int64_t n_nodes, int64_t n_edges, const int64_t* edges, const double* coords,
                        const double* coef, int64_t n_triples, const int64_t* triples, double EI, int mem,
                        void* stream, int64_t* row_ptr, int32_t* col, double* val, int64_t cap_nnz,
                        int64_t* nnz_out);

/* build_network_operator -- the free-dof operator of a network problem.
 *
 * Section 3: with Dirichlet dofs D (values g) and free dofs I, the solver
 * works on A = K_II and the lifted right-hand side b = f_I - K_ID g_D.
 * dim in {2, 3}; ndof in {1, 3}; coords [n_nodes*dim] inside
 * Omega = [0, domain_hi[0]] x ... ; K given as CSR on all n_nodes*ndof dofs
 * (row_ptr [n_dof+1] int64, col_idx [nnz] int32 sorted ascending per row,
 * vals [nnz]), symmetric; dirichlet_dofs [n_dirichlet] strictly ascending.
 * Errors: BAD_INPUT (unsorted/out-of-range indices, asymmetric K_II beyond
 * 1e-12 relative, non-positive diagonal, coordinates outside Omega).
 */
int build_network_operator(int dim, int ndof, int64_t n_nodes, const double* coords,
                           const int64_t* row_ptr, const int32_t* col_idx, const double* vals,
                           int64_t n_dirichlet, const int64_t* dirichlet_dofs,
                           const double* domain_hi, int mem, void* stream, spnet_op_t* out);

/* setup_preconditioner -- the two-level additive Schwarz preconditioner B.
 *
 * Section 2.3 / 4.1.  H must divide every side length (l_i / H integral).
 * gamma_faces [ndof] (host): per component, the bitmask of box faces on which
 * that component is Dirichlet (bit 2*axis for x_axis = 0, bit 2*axis+1 for
 * x_axis = l_axis); mesh nodes on those faces carry no coarse dof.  Coarse
 * basis functions are truncated to free dofs; a function that vanishes at
 * every free dof of its component is dropped.  When the truncated functions
 * are linearly dependent (A_0 singular), the coarse solve works on a basis of
 * their span V_H: in coarse-dof order, a function whose pivot in the
 * elimination of A_0 is at most 1e-8 times its diagonal entry of A_0 lies in
 * the span of the functions before it and is left out
 * (spnet_pc_info.coarse_dropped); P_0 is unchanged.  In mixed precision A_0
 * is inverted in FP32 unless a pivot falls to 1e-3 of its diagonal entry or
 * below, in which case the inverse is formed in FP64 and rounded.  opts may be
 * NULL (defaults).  Errors: BAD_H, NOT_SPD (a local pivot <= 0), UNSUPPORTED
 * (a star beyond 65535 dofs), NO_MEMORY, BAD_INPUT (an unknown option; or, with
 * support patches or P1 element patches, a free dof that lies in no star, which
 * would leave B singular there: take stars at every mesh node).
 */
int setup_preconditioner(spnet_op_t op, double H, const int* gamma_faces,
                         const spnet_options* opts, spnet_pc_t* out);

/* pcg_solve -- preconditioned conjugate gradients for nrhs right-hand sides.
 *
 * Section 4.2.  f [nrhs*n_dof] (values at Dirichlet dofs ignored),
 * g [nrhs*n_dirichlet] Dirichlet values in the order of dirichlet_dofs,
 * x [nrhs*n_dof]: on entry the initial guess if use_x0 (free dofs only), on
 * exit u_hat = u + g on all dofs.  Stops when ||r||_2 <= rtol ||b||_2 on the
 * recursive residual, then recomputes b - A x in FP64 and restarts from it
 * (at most max_restarts times) if it is above the tolerance.  stats [nrhs]
 * is host memory (may be NULL).  Returns NO_CONVERGENCE if any right-hand
 * side misses rtol within maxit steps (x is still written), BAD_INPUT if a
 * right-hand side's lifted data b = f_I - K_ID g or its initial residual is
 * not finite (a NaN or Inf at a free dof of f, in g, or in x0).
 */
int pcg_solve(spnet_op_t op, spnet_pc_t pc, int nrhs, const double* f, const double* g,
              double* x, int use_x0, double rtol, int maxit, int mem, spnet_stats* stats);

int spnet_op_destroy(spnet_op_t op);
int spnet_pc_destroy(spnet_pc_t pc);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of solve requests.
 *
 * The paper solves one network at a time; this is the service around the
 * same solver (assembly, build_network_operator, setup_preconditioner,
 * pcg_solve per request).  A server runs up to max_inflight requests at once,
 * each on its own CUDA stream and host thread; requests wait in submission
 * order and are admitted when a slot is free and the device memory the
 * request is estimated to need fits the budget (the free device memory at
 * creation less reserve_bytes, less the estimates of the running requests).
 * The admitted requests' work overlaps on the GPU.  Every kernel reduces in a
 * fixed order, so a request's result does not depend on what else runs.
 * ------------------------------------------------------------------------- */
typedef struct spnet_server_s* spnet_server_t;

typedef struct {
  int model;                     /* SPNET_MODEL_SCALAR or SPNET_MODEL_TRUSS3 */
  int dim;                       /* 2 or 3 */
  int64_t n_nodes, n_edges;
  const int64_t* edges;          /* [2*n_edges] node ids (i, j) */
  const double* coef;            /* [n_edges] edge coefficients (as spnet_assemble) */
  const double* dirs;            /* [3*n_edges] unit edge directions (TRUSS3), else NULL */
  const double* coords;          /* [n_nodes*dim] */
  double domain_hi[3];           /* Omega = [0, domain_hi[0]] x ... */
  int64_t n_dirichlet;
  const int64_t* dirichlet_dofs; /* [n_dirichlet] strictly ascending */
  int nrhs;                      /* right-hand sides of this request, >= 1 */
  const double* f;               /* [nrhs*n_dof] */
  const double* g;               /* [nrhs*n_dirichlet] Dirichlet values */
  double* x;                     /* [nrhs*n_dof] out: u_hat = u + g on all dofs */
  double H;                      /* coarse mesh width (as setup_preconditioner) */
  int gamma_faces[3];            /* per component (first ndof used), as setup_preconditioner */
  spnet_options opts;            /* as setup_preconditioner */
  double rtol;                   /* relative residual target */
  int maxit;
  int reserved[7];
} spnet_request;

typedef struct {
  int status;               /* SPNET_OK, or the error code of the failed step */
  int iterations;           /* largest CG step count over the request's right-hand sides */
  double relres;            /* largest recomputed relative residual */
  double queue_ms;          /* submission -> admission (host clock) */
  double latency_ms;        /* submission -> solutions in host memory (host clock) */
  double device_start_ms;   /* device time of the request's first and last work, from */
  double device_end_ms;     /*   an origin fixed when the server was created (CUDA events) */
  char message[256];        /* the error message when status != SPNET_OK */
} spnet_result;

/* spnet_server_create -- start max_inflight (1..64) workers on the current device.  The
 * memory budget of the running requests is the device's free memory now, less
 * reserve_bytes (NO_MEMORY if that is not positive). */
int spnet_server_create(int max_inflight, int64_t reserve_bytes, spnet_server_t* out);
/* spnet_server_submit -- queue a request (host arrays, borrowed until spnet_server_wait or
 * spnet_server_poll has returned its result); *ticket identifies it.  Errors: BAD_INPUT
 * (malformed request), NO_MEMORY (its estimated peak device memory, spnet_server_estimate,
 * exceeds the server's budget: it could never be admitted; nothing is queued). */
int spnet_server_submit(spnet_server_t server, const spnet_request* request, int64_t* ticket);
/* spnet_server_wait -- block until the request is done; its result (the solutions are in
 * request->x).  A request that failed reports its error in result->status/message. */
int spnet_server_wait(spnet_server_t server, int64_t ticket, spnet_result* result);
/* spnet_server_poll -- the non-blocking form of spnet_server_wait: *done = 1 and the result
 * (the ticket is then retired) if the request has finished, else *done = 0. */
int spnet_server_poll(spnet_server_t server, int64_t ticket, spnet_result* result, int* done);
/* spnet_server_cancel -- withdraw a request that is still queued: *cancelled = 1 and its
 * result (wait/poll) reports SPNET_ERR_CANCELLED; a request already admitted runs to its
 * end (*cancelled = 0).  Errors: BAD_INPUT (unknown ticket). */
int spnet_server_cancel(spnet_server_t server, int64_t ticket, int* cancelled);
/* spnet_server_estimate -- the peak device bytes admission charges for a request (the
 * operator and its copies of K, star factors and solve windows, the dense A_0 and its
 * inverse, the PCG vectors and blocks).  Host only. */
int spnet_server_estimate(const spnet_request* request, int64_t* bytes);
/* spnet_server_budget -- the device bytes the server's running requests may hold. */
int spnet_server_budget(spnet_server_t server, int64_t* bytes);
/* spnet_server_destroy -- finish every queued request, stop the workers, free the server. */
int spnet_server_destroy(spnet_server_t server);

/* The tuner.  setup_preconditioner times, once per device and size class, the warps per
 * block of the one-vector star solve (unless spnet_options.star_map fixes it), the lanes
 * per row of the SpMV (operators of 65536 free dofs or more) and the right-hand sides per
 * warp of the batched star solve (batch_rhs >= 4), on the preconditioner's own data, and
 * keeps the choices in a process-wide cache.  The last two change the order of sums, so
 * every set-up of a class uses the one measured value (a set-up meeting a class being
 * measured waits for it).  The cache can be saved and loaded, so that another process takes
 * the same choices without measuring: a text file of lines
 * "device<TAB>kind<TAB>c0,c1,c2,c3<TAB>value" (device: name, SM count, compute capability).
 * spnet_tune_cache_load  add the lines of a file to the cache.  Errors: BAD_INPUT (unreadable
 *                        file or malformed line; nothing is added then).
 * spnet_tune_cache_save  write the cache's measured entries (all devices) to a file.
 * spnet_tune_cache_clear forget every measured entry and the counts.
 * spnet_tune_counts      choices measured, and choices taken from the cache, since the clear. */
int spnet_tune_cache_load(const char* path);
int spnet_tune_cache_save(const char* path);
int spnet_tune_cache_clear(void);
int spnet_tune_counts(int64_t* measured, int64_t* reused);

/* spnet_last_error -- copy the calling thread's last error message (NUL-terminated). */
int spnet_last_error(char* buf, size_t len);

int spnet_op_get_info(spnet_op_t op, spnet_op_info* info);
int spnet_pc_get_info(spnet_pc_t pc, spnet_pc_info* info);

/* The steps of one preconditioner application, for checking each one on its
 * own.  Vectors on the free dofs are in ascending-dof order ("free order");
 * coarse vectors are in coarse-dof order (mesh node ascending, lexicographic
 * with axis 0 fastest, then component).
 *
 * spnet_spmv          y = A x                         (Section 3, A = K_II)
 * spnet_pc_apply      z = B r                         (Section 4.1-4.2)
 * spnet_pc_restrict   r_c = R_0 r                     (Section 2.3: Q1 values at free dofs)
 * spnet_pc_coarse     z_c = A_0^{-1} r_c              (P_0, eq. defPj)
 * spnet_pc_prolong    z = R_0^T z_c
 * spnet_pc_stars      z = sum_j E_j A_j^{-1} E_j^T r  (P_j, eq. defPj)
 */
int spnet_spmv(spnet_op_t op, const double* x, double* y, int mem);
int spnet_pc_apply(spnet_pc_t pc, const double* r, double* z, int mem);
int spnet_pc_restrict(spnet_pc_t pc, const double* r, double* rc, int mem);
int spnet_pc_coarse(spnet_pc_t pc, const double* rc, double* zc, int mem);
int spnet_pc_prolong(spnet_pc_t pc, const double* zc, double* z, int mem);
int spnet_pc_stars(spnet_pc_t pc, const double* r, double* z, int mem);

/* spnet_pc_apply_batch -- z_j = B r_j for k right-hand sides at once (1 <= k <= 32),
 * the form of spnet_pc_apply that pcg_solve uses when it steps right-hand sides
 * together (Sections 4.1-4.2 applied to each r_j on its own).  r, z [k*n_free]:
 * one right-hand side after another, each in free order; host or device memory
 * by mem.  which: 0 the whole of B; 1 the coarse term R_0^T A_0^{-1} R_0 r only;
 * 2 the star term sum_j E_j A_j^{-1} E_j^T r only.  Where the largest star's
 * solve vector for k right-hand sides does not fit a block's shared memory, the
 * right-hand sides go in several passes of the widest block that does.  Errors:
 * BAD_INPUT (null pointer, k, which or mem out of range), UNSUPPORTED (the
 * largest star alone exceeds a block's shared memory), CUDA.
 */
int spnet_pc_apply_batch(spnet_pc_t pc, int k, const double* r, double* z, int which, int mem);

/* spnet_pc_export -- copy set-up data to host memory (for inspection).
 * what: SPNET_EXPORT_ELEMENTS   int32 [n_free]     linear host element of each free dof
 *       SPNET_EXPORT_Q1         double [n_free*2^d] Q1 values, free-dof major
 *       SPNET_EXPORT_COARSE_MAP int32 [n_mesh*ndof] coarse index of (mesh node, component), -1 if none
 *       SPNET_EXPORT_STAR_SIZES int32 [n_stars]    dofs of each star (stars in mesh order)
 *       SPNET_EXPORT_STAR_MESH  int32 [n_stars]    mesh node of each star
 *       SPNET_EXPORT_A0         double [m0*m0]     the Galerkin matrix A_0 (row-major)
 *       SPNET_EXPORT_STAR_LEVELS int32 [n_stars]   level count of each star's local solve
 *       SPNET_EXPORT_STAR_CORE  int32 [n_stars]    nodes of the dense block that ends each star's
 *                                                  elimination (0: none)
 * bytes must be at least the size listed.
 */
#define SPNET_EXPORT_ELEMENTS 0
#define SPNET_EXPORT_Q1 1
#define SPNET_EXPORT_COARSE_MAP 2
#define SPNET_EXPORT_STAR_SIZES 3
#define SPNET_EXPORT_STAR_MESH 4
#define SPNET_EXPORT_A0 5
#define SPNET_EXPORT_STAR_LEVELS 6
#define SPNET_EXPORT_STAR_CORE 7
int spnet_pc_export(spnet_pc_t pc, int what, void* host_buf, size_t bytes);

/* spnet_pc_restrict_static -- r_c = R_0 r, exactly as spnet_pc_restrict, but the
 * call allocates no memory at all.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory at the time of
 * the call -- hosts whose device memory is all reserved up front by another
 * allocator (a framework's caching pool that has taken the whole GPU), and
 * latency-bound loops that must not enter cudaMalloc, which can synchronise
 * the device and take an unbounded time.
 *
 * r (device, free order, n_free doubles) and rc (device, coarse order, m0
 * doubles) are the caller's, on the preconditioner's device, which must be
 * the current device (else SPNET_ERR_BAD_INPUT).  The scratch -- the
 * Q1-weighted sums of r at the 2^d corners of every element, n_elem * 2^d *
 * ndof doubles -- lives in one fixed array of 2^18 doubles (2 MiB) inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  Meshes that need more corner sums are rejected with
 * SPNET_ERR_UNSUPPORTED.  The first call on a device looks the array's device
 * address up (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  All calls share the one array and it keeps
 * the last call's contents: calls whose work overlaps on the GPU (other
 * threads, other streams, several preconditioners) race and must be
 * serialised by the caller.  Every entry of the array that a call reads is
 * written earlier in the same call, so nothing has to be cleared between
 * calls.  Runs on the operator's stream and returns when rc is complete. */
int spnet_pc_restrict_static(spnet_pc_t pc, const double* r, double* rc);

/* spnet_pc_record_iterates -- keep the PCG iterates of later solves (the rate
 * experiments of Section 6: the K-norm error |u - u^(l)|_K after every step l,
 * eq. conv_rate).  While set, every spnet_pcg_solve that takes its right-hand
 * sides one at a time (batch_rhs = 1) writes, for each right-hand side in turn,
 * u^(l) restricted to the free dofs (free order, n_free doubles) to
 * buf + l * n_free for the step counts l = 0 (the initial guess), 1, 2, ...
 * below max_iterates; later steps are not kept, and the next right-hand side
 * writes over the previous one's.  Steps keep counting across restarts.
 * buf: device memory of the preconditioner's device, the caller's, at least
 * max_iterates * n_free doubles, 8-byte aligned.  buf = NULL with
 * max_iterates = 0 stops recording.  Recording runs the iterations as separate
 * launches (not the chunked CUDA graph), one more kernel per step.  Errors:
 * BAD_INPUT (null pc; buf NULL with max_iterates > 0 or the reverse;
 * max_iterates < 0; buf not device memory of the preconditioner's device;
 * max_iterates * n_free beyond 2^62). */
int spnet_pc_record_iterates(spnet_pc_t pc, double* buf, int64_t max_iterates);

/* Instrumentation (process-wide; not part of the paper's method).
 * spnet_launch_count   kernels the library has launched since it was loaded.
 * spnet_profile_enable 1: time every launch of the kernels below with CUDA
 *                      events recorded on the launching stream; 0: stop.
 * spnet_profile_read   launches and total milliseconds of one kernel since the
 *                      last reset (reading waits for the recorded events).
 * spnet_profile_reset  clear the accumulated timings. */
#define SPNET_KERNEL_SPMV 0
#define SPNET_KERNEL_UPDATE 1
#define SPNET_KERNEL_RESTRICT 2
#define SPNET_KERNEL_STARS 3
#define SPNET_KERNEL_COARSE 4
#define SPNET_KERNEL_COMBINE 5
#define SPNET_KERNEL_DIRECTION 6
#define SPNET_KERNEL_STAR_SYMBOLIC 7
#define SPNET_KERNEL_STAR_NUMERIC 8
#define SPNET_KERNEL_SWEEP 9
#define SPNET_KERNEL_GALERKIN 10
#define SPNET_KERNEL_COUNT 11
int spnet_launch_count(int64_t* count);
int spnet_profile_enable(int on);
int spnet_profile_read(int kernel, int64_t* launches, double* total_ms);
int spnet_profile_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* SPNET_H */
