// Internal declarations shared by the translation units of libspnet.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/spnet.h"

namespace spnet {

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
const std::string& last_error();
int fail(int code, const std::string& msg);

struct Status {
  int code = SPNET_OK;
  std::string msg;
};

#define SPNET_CUDA_TRY(expr)                                                          \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) {                                                          \
      return ::spnet::fail(_e == cudaErrorMemoryAllocation ? SPNET_ERR_NO_MEMORY      \
                                                           : SPNET_ERR_CUDA,          \
                           std::string(#expr) + ": " + cudaGetErrorString(_e));       \
    }                                                                                 \
  } while (0)

#define SPNET_TRY(expr)           \
  do {                            \
    int _rc = (expr);             \
    if (_rc != SPNET_OK) return _rc; \
  } while (0)

// device-side error flags (bitmask in a device int)
enum : int {
  FLAG_BAD_INPUT = 1,
  FLAG_NOT_SPD = 2,
  FLAG_ASYM = 4,
  FLAG_POOL = 8,        // star factor pool too small (retry with a larger pool)
  FLAG_STAR_BIG = 16,   // star or dense core beyond the scratch capacity
  FLAG_NONFINITE = 32,
  FLAG_OUT_OF_BOX = 64,
  FLAG_UNSORTED = 128,
  FLAG_COARSE_SPD = 256,
  FLAG_UNCOVERED = 512,  // a free dof in no star (a patch test in use and too few stars)
};

// ---------------------------------------------------------------------------
// stream-ordered device buffers
// ---------------------------------------------------------------------------
struct DevArena {
  cudaStream_t stream = 0;
  std::vector<void*> ptrs;
  std::vector<int64_t> sizes;
  int64_t bytes = 0;  // bytes currently held
  int alloc(void** p, size_t n);
  template <class T>
  int get(T** p, size_t count) {
    return alloc(reinterpret_cast<void**>(p), count * sizeof(T));
  }
  void release(void* p);
  void free_all();
};

// ---------------------------------------------------------------------------
// operator and preconditioner handles
// ---------------------------------------------------------------------------
struct Csr {
  int64_t n = 0, nnz = 0;
  int64_t* ptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};

// PCG scalars on the device; each field has one writer per kernel (the last
// block of the kernel that finishes its reduction)
struct Scal {
  double rz, pq, rr, bb, alpha, beta, rr_true, rtol;
  int maxit, iter, done, restarts;
  unsigned cnt[4];  // arrival counters of the last-block reductions
};

}  // namespace spnet
struct spnet_pc_s;
namespace spnet {
// the tuner's cache (tune.cu): choices per device, kind and size class
enum : int { TUNE_STAR_MAP = 0, TUNE_SPMV_LANES = 1, TUNE_BATCH_JW = 2, TUNE_KINDS = 3 };
struct TuneClass {
  int c[4];
};
// 1 and *value: the class's choice is known; 0: the caller measures it and reports it with
// tune_end (value 0: failed).  Waits while another set-up measures the class.
int tune_begin(int kind, const TuneClass& c, int* value);
void tune_end(int kind, const TuneClass& c, int value);
int tune_peek(int kind, const TuneClass& c, int* value);  // 1 and *value if known; never waits
int assemble_beam(int64_t n_nodes, int64_t n_edges, const int64_t* edges, const double* coords,
                  const double* coef, int64_t n_tri, const int64_t* tri, double EI, int mem, cudaStream_t s,
                  int64_t* row_ptr, int32_t* col, double* val, int64_t cap_nnz, int64_t* nnz_out);
int spmv_grid(const spnet_pc_s* pc, int lanes);
int spmv_lanes_tune(spnet_pc_s* pc);
int batch_jw_tune(spnet_pc_s* pc);
int half_octave(double x);

}  // namespace spnet

struct spnet_op_s {
  int dim = 0, ndof = 0;
  int64_t n_nodes = 0, n_dof = 0, n_free = 0, n_dir = 0;
  double domain[3] = {1, 1, 1};
  cudaStream_t stream = 0;
  int device = 0;               // CUDA device current when the operator was built
  bool own_stream = false;      // created by the library (the caller passed stream 0)
  spnet::DevArena mem;
  double* coords = nullptr;     // [n_nodes*dim]
  int64_t* dir_dofs = nullptr;  // [n_dir]
  int64_t* free_dofs = nullptr; // [n_free]
  int64_t* free_of = nullptr;   // [n_dof]: free index, or -(position in dir_dofs) - 2
  spnet::Csr ff, fd;            // K_II, K_ID
  int* dflags = nullptr;
  double* spmv_tmp = nullptr;   // [2*n_free] scratch for spnet_spmv on host arrays
  int refcount = 0;
};

struct spnet_pc_s {
  spnet_op_s* op = nullptr;
  spnet::DevArena mem;
  int precision = SPNET_PREC_MIXED, star_set = SPNET_STARS_INTERIOR, flexible = 1, max_restarts = 2;
  int batch_rhs = 1;            // right-hand sides pcg_solve steps together
  int star_map = 0;             // warps per block of the star solve: 0 tuned per size class
  int patch = SPNET_PATCH_ELEMENT;  // dofs a star holds (SPNET_PATCH_*)
  int coarse_space = SPNET_COARSE_Q1;  // SPNET_COARSE_*
  // The star kernels' patch test: a dof is off the star of the mesh node at its host element's
  // corner c when patch_w[c][dof] == 0 (star_rule SUPPORT) -- the basis values for support
  // patches, the vertex indicator of the host simplex for P1 element patches -- or never
  // (star_rule ELEMENT: Q1 element patches).
  int star_rule = SPNET_PATCH_ELEMENT;
  double* patch_w = nullptr;    // [nc][N]: q1w, or the vertex indicator (P1 element patches)
  double* rec_buf = nullptr;    // spnet_pc_record_iterates: the caller's [rec_max*N], free order
  int64_t rec_max = 0;
  int d = 0, ndof = 1, nc = 4;  // nc = 2^d corners
  int gamma[3] = {0, 0, 0};     // Dirichlet face bitmask per component
  int nH[3] = {1, 1, 1};
  int n_elem = 0, n_mesh = 0;
  double H = 0;
  int64_t N = 0;  // free dofs
  // permutation: pc position <-> free index
  int32_t* perm = nullptr;     // [N] free index at pc position
  int32_t* iperm = nullptr;    // [N]
  int32_t* elem_of = nullptr;  // [N] element of pc position
  int8_t* comp_of = nullptr;   // [N]
  int32_t* elem_ptr = nullptr; // [n_elem+1]
  double* q1w = nullptr;       // [nc][N]
  double* xi = nullptr;        // [d*N] local coordinates of each dof in its element (axis-major)
  float* xi32 = nullptr;       // [d*N] the same in FP32 (mixed precision: restriction and prolongation in FP32)
  spnet::Csr K;                // A in pc order
  // coarse space
  int m0 = 0;
  int coarse_dropped = 0;      // coarse functions left out as dependent on the others
  int32_t* cidx = nullptr;     // [n_mesh*ndof]
  void* ctiles = nullptr;      // A_0^{-1} (float or double by precision): its upper 128 x 128 tiles, packed
  void* cpart = nullptr;       // [nt*nt*CT] per row block and tile column: partial products
  int ctiles_n = 0;            // nt: tiles per dimension
  int32_t* rtab = nullptr;     // [m0*8] offsets of the corner sums that make up each r_c entry
  double* A0 = nullptr;        // [m0*m0] copy of A_0 if m0 <= A0_KEEP
  // stars
  int S = 0, max_star = 0, max_levels = 0;
  int64_t sum_s = 0, factor_nnz = 0, total_levels = 0;
  int32_t* star_mesh = nullptr;    // [S]
  int32_t* star_of_mesh = nullptr; // [n_mesh]
  int64_t* star_ptr = nullptr;     // [S+1]
  int32_t* elem_star_off = nullptr;// [n_elem*nc], -1 if no star at that corner
  char* pool = nullptr;
  int64_t pool_bytes = 0;
  int64_t* star_off = nullptr;     // [S] byte offset of each star's factor blob
  int32_t* star_n = nullptr;       // [S]
  int32_t* star_lev = nullptr;     // [S]
  int32_t* star_nnz = nullptr;     // [S]
  int32_t* star_core = nullptr;    // [S] nodes of the dense block that ends each star's elimination
  // k-right-hand-side solves (FP32) of stars whose dense block is solved by panels on tensor cores
  int panels = 1;                  // build them (spnet_options.panels)
  int panel_stars = 0;             // stars solved that way
  void* bhdr = nullptr;            // [S] headers of the k-right-hand-side solve (null: none)
  char* brec = nullptr;            // their window records
  float* coreL = nullptr;          // the dense blocks' tiles in MMA fragment order
  int64_t panel_bytes = 0;         // bytes of brec and coreL
  // solve windows: per-star header (80 B), inverse permutation, window records
  void* shdr = nullptr;            // [S] headers
  uint16_t* iperm_star = nullptr;  // [sum_s] local index -> elimination position, at star_ptr
  char* srec = nullptr;            // [n_entries] window records (208 B FP32, 336 B FP64)
  int64_t n_entries = 0;           // window records of all stars
  int64_t stream_bytes = 0;        // bytes one solve reads from headers, permutations and records
  int solve_wpb = 0;               // warps (stars) per block of the solve
  int solve_blocks = 0;            // blocks of the solve (a multiple of the SM count)
  size_t solve_smem = 0;           // its dynamic shared memory per block
  int32_t* sorder = nullptr;       // [solve_blocks*solve_wpb] star of each warp slot, -1: idle
  int32_t* star_desc = nullptr;    // [S] stars by solve cost, largest first
  std::vector<double> star_cost;   // [S] host: estimated solve cost of each star
  std::vector<int32_t> star_ord;   // [S] host: stars by cost, largest first
  int solve_wpb_max = 0;           // most warps per block the shared-memory budget holds
  // work vectors (pc order)
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *b = nullptr;
  double* r2 = nullptr;            // second residual buffer (the iterations alternate)
  double *rc = nullptr, *zc = nullptr, *partial = nullptr, *vtmp = nullptr;
  void* w = nullptr;               // [sum_s] star results in the solve precision (float or double)
  double* epart = nullptr;         // [n_elem*nc*ndof] Q1-weighted corner sums of r
  int32_t* ecoarse = nullptr;      // [n_elem*nc*ndof] coarse index at each corner (-1: none)
  int64_t* estar = nullptr;        // [n_elem*nc] base of the element's entries in w (-1: no star)
  spnet::Scal* scal = nullptr;
  cudaGraphExec_t graph_exec = nullptr;  // a chunk of PCG iterations
  cudaStream_t side = nullptr;     // second stream of the graph (star solves)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int graph_launches = 0;
  int G = 0;         // reduction grid
  int PG = 0;        // stride of the partial-sum slots (max blocks of a reducing kernel)
  int spmv_lanes = 1;
  int batch_jw = 0;                // right-hand sides per warp of the batched star solve (0: by k)
  int spmv_blocks = 1;             // grid of the SpMV of an iteration (one pass over the rows)
  double* pspmv = nullptr;         // [spmv_blocks] its partial dot products
  double setup_ms = 0;
};

namespace spnet {

// ---------------------------------------------------------------------------
// the Cartesian mesh T_H: elements numbered lexicographically with axis 0
// fastest, mesh nodes likewise over (n_a + 1) per axis, corner c of an element
// has bit a set when it sits at the upper end of axis a
// ---------------------------------------------------------------------------
struct Mesh {
  int d, nc;
  int n[3];         // elements per axis
  int simplex = 0;  // 1: P1 on the Kuhn simplices of the boxes (SPNET_COARSE_P1)
};

__device__ __forceinline__ void elem_multi(const Mesh& m, int e, int* ex) {
  ex[0] = e % m.n[0];
  int t = e / m.n[0];
  ex[1] = t % m.n[1];
  ex[2] = m.d == 3 ? t / m.n[1] : 0;
}

// mesh node at corner c of element e (corner bit a = offset along axis a)
__device__ __forceinline__ int mesh_of(const Mesh& m, int e, int c) {
  int ex[3];
  elem_multi(m, e, ex);
  int k = ex[0] + (c & 1);
  k += (m.n[0] + 1) * (ex[1] + ((c >> 1) & 1));
  if (m.d == 3) k += (m.n[0] + 1) * (m.n[1] + 1) * (ex[2] + ((c >> 2) & 1));
  return k;
}

__device__ __forceinline__ void mesh_multi(const Mesh& m, int k, int* km) {
  km[0] = k % (m.n[0] + 1);
  int t = k / (m.n[0] + 1);
  km[1] = t % (m.n[1] + 1);
  km[2] = m.d == 3 ? t / (m.n[1] + 1) : 0;
}

// element e' = k - 1 + c' around mesh node k, or -1 outside the mesh
__device__ __forceinline__ int elem_around(const Mesh& m, const int* km, int cp) {
  int e = 0, stride = 1;
  for (int a = 0; a < m.d; ++a) {
    int ea = km[a] - 1 + ((cp >> a) & 1);
    if (ea < 0 || ea >= m.n[a]) return -1;
    e += ea * stride;
    stride *= m.n[a];
  }
  return e;
}

inline Mesh mesh_of_pc(const spnet_pc_s* pc) {
  Mesh m;
  m.d = pc->d;
  m.nc = pc->nc;
  for (int a = 0; a < 3; ++a) m.n[a] = pc->nH[a];
  m.simplex = pc->coarse_space == SPNET_COARSE_P1 ? 1 : 0;
  return m;
}

constexpr int RED_BLOCK = 256;
constexpr int A0_KEEP = 2048;

// util.cu
enum KernelId {
  KID_SPMV = 0, KID_UPDATE, KID_RESTRICT, KID_STARS, KID_COARSE, KID_COMBINE, KID_DIRECTION,
  KID_STAR_SYMBOLIC, KID_STAR_NUMERIC, KID_SWEEP, KID_GALERKIN, KID_COUNT
};
void note_launch();
void add_launches(long long n);
long long launch_count();
bool profiling_on();
struct ProfScope {
  int id;
  cudaStream_t s;
  cudaEvent_t a{}, b{};
  bool active = false;
  ProfScope(int id, cudaStream_t s);
  ~ProfScope();
};
void profile_enable(int on);
void profile_read(int id, long long* n, double* ms);
void profile_reset();
int scan_exclusive(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s, DevArena& mem);
int scan_exclusive64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, DevArena& mem);
int copy_in(const void* src, void* dst, size_t bytes, int mem, cudaStream_t s);
int copy_out(const void* src, void* dst, size_t bytes, int mem, cudaStream_t s);
int check_flags(int* dflags, cudaStream_t s, const char* where);
void fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s);
int num_sms();
double elapsed_ms(cudaEvent_t a, cudaEvent_t b);

// operator.cu
void launch_spmv(const Csr& A, const double* x, double* y, double* partial_pq, int G, int lanes,
                 const int* done, cudaStream_t s);
int choose_spmv_lanes(const Csr& A);

// setup.cu
int pc_setup_structure(spnet_pc_s* pc);
int pc_galerkin(spnet_pc_s* pc, double* A0_dense);

// starfact.cu
int pc_factor_stars(spnet_pc_s* pc);
// star solves for k <= 32 right-hand sides at once (R, W: [dofs][k]); W in the solve precision
int launch_star_batch(spnet_pc_s* pc, const double* R, int k, void* W, const int* done, cudaStream_t s);
// the largest block width (a power of two <= 32) whose star solve fits a block's shared memory
int star_batch_max_k(const spnet_pc_s* pc);
// the star solve's mapping (warps per block): fixed by the options, or tuned per size class
int star_map_tune(spnet_pc_s* pc);
// coarse solve for k <= 32 right-hand sides at once: ZC [m0][k] from the corner sums EP [entries][k]
size_t coarse_batch_part_bytes(const spnet_pc_s* pc, int k);
int launch_coarse_batch(spnet_pc_s* pc, const double* EP, int k, double* ZC, void* part, const int* done,
                        cudaStream_t s);
// stars on r, or (q set: a PCG step) on r - alpha q with alpha from the SpMV's partials
void launch_star_solve(spnet_pc_s* pc, const double* r, const double* q, const spnet::Scal* sc, const int* done,
                       cudaStream_t s);

// coarse.cu
int pc_coarse_invert(spnet_pc_s* pc, double* A0_dense);
int coarse_gemv_prepare(spnet_pc_s* pc);
void launch_coarse_apply(spnet_pc_s* pc, const double* rc, double* zc, const int* done,
                         cudaStream_t s);

// pcg.cu
void launch_restrict(spnet_pc_s* pc, double* rc, const int* done, cudaStream_t s);
void launch_combine(spnet_pc_s* pc, const double* r, double* z, int with_coarse, int with_stars,
                    int dots, cudaStream_t s, int exact = 0);
int pc_restrict_free(spnet_pc_s* pc, const double* r_free, double* rc);
int pc_elem_tables(spnet_pc_s* pc);
int pc_apply_free(spnet_pc_s* pc, const double* r_free_dev, double* z_free_dev, int which);
void to_pc(spnet_pc_s* pc, const double* free_vec, double* pc_vec);
void from_pc(spnet_pc_s* pc, const double* pc_vec, double* free_vec);
int export_item(spnet_pc_s* pc, int what, void* host_buf);
int pcg_run(spnet_op_s* op, spnet_pc_s* pc, int nrhs, const double* f, const double* g, double* x,
            int use_x0, double rtol, int maxit, int mem, spnet_stats* stats);
__global__ void k_build_rhs(int64_t N, const int32_t* perm, const int64_t* free_dofs, const double* f,
                            const int64_t* fdp, const int32_t* fdc, const double* fdv, const double* g,
                            double* b);
__global__ void k_x0_from_dofs(int64_t N, const int32_t* perm, const int64_t* free_dofs, const double* x,
                               double* xp);
__global__ void k_expand(int64_t n_dof, const int64_t* free_of, const int32_t* iperm, const double* xp,
                         const double* g, double* out);
__global__ void k_residual(int64_t N, const double* b, const double* q, double* r, double* partial,
                           double* out, unsigned* cnt);

// batch.cu: k (2..32) right-hand sides stepped together; device arrays f [k][n_dof],
// g [k][n_dir], x [k][n_dof]; stats [k] host
int pcg_batch_run(spnet_op_s* op, spnet_pc_s* pc, int k, const double* f, const double* g, double* x,
                  int use_x0, double rtol, int maxit, spnet_stats* stats);
// z_j = B r_j (which 0), the coarse term (1) or the star term (2) for k <= 32 residuals;
// r, z device [k][n_free] in free order
int pc_apply_batch_free(spnet_pc_s* pc, int k, const double* r, double* z, int which);

// Butterfly reduce-scatter of K per-lane values (K a power of two, K <= 32):
// K-1 + log2(32/K) shuffles instead of 5K.  Afterwards lane L holds the warp
// total of index rs_index<K>(L) if rs_writer<K>(L).  Fixed order: deterministic.
template <int K, class T>
__device__ __forceinline__ T reduce_scatter(T (&v)[K], int lane) {
#pragma unroll
  for (int h = K / 2, bit = 16; h >= 1; h >>= 1, bit >>= 1) {
    const bool upper = (lane & bit) != 0;
#pragma unroll
    for (int t = 0; t < h; ++t) {
      const T send = upper ? v[t] : v[t + h];
      const T recv = __shfl_xor_sync(0xffffffffu, send, bit);
      v[t] = (upper ? v[t + h] : v[t]) + recv;
    }
  }
  T s = v[0];
#pragma unroll
  for (int bit = 16 / K; bit >= 1; bit >>= 1) s += __shfl_xor_sync(0xffffffffu, s, bit);
  return s;
}

template <int K>
__device__ __forceinline__ int rs_index(int lane) {
  int idx = 0;
#pragma unroll
  for (int h = K / 2, bit = 16; h >= 1; h >>= 1, bit >>= 1)
    if (lane & bit) idx += h;
  return idx;
}

template <int K>
__device__ __forceinline__ bool rs_writer(int lane) {
  return (lane & (32 / K - 1)) == 0;
}

// Programmatic dependent launch.  A kernel of the iteration lets the next
// kernel of its stream launch as soon as all of its blocks run
// (pdl_trigger), and waits, before it reads anything the previous kernel
// wrote, until that kernel has finished and its memory is visible (pdl_wait).
// Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// launch with programmatic stream serialization: the kernel may start while
// the previous kernel of the stream finishes (it must call pdl_wait first)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// P1 values on the Kuhn simplex that holds local coordinates t (Remark 2.1): with pi the
// axes in order of non-increasing t (ties: the smaller axis first), the corner with bits
// {pi(0), .., pi(j-1)} gets t_pi(j-1) - t_pi(j) (t_pi(-1) = 1, t_pi(d) = 0), the other
// corners zero; the same differences, in the same order, as the stored P1 values.
// pi by insertion with strict comparisons (a stable sort); the values are placed with
// selects against compile-time corners, so nothing is indexed at run time.
template <int NC, class CT>
__device__ __forceinline__ void p1_sorted(const CT (&t)[3], CT& a0, CT& a1, CT& a2, int& b0, int& b1, int& b2) {
  constexpr int D = NC == 4 ? 2 : 3;
  a0 = t[0];
  a1 = t[1];
  a2 = D == 3 ? t[2] : CT(0);
  b0 = 1;
  b1 = 2;
  b2 = 4;
  if (a1 > a0) {
    const CT x = a0; a0 = a1; a1 = x;
    const int y = b0; b0 = b1; b1 = y;
  }
  if (D == 3 && a2 > a1) {
    { const CT x = a1; a1 = a2; a2 = x; }
    { const int y = b1; b1 = b2; b2 = y; }
    if (a1 > a0) {
      const CT x = a0; a0 = a1; a1 = x;
      const int y = b0; b0 = b1; b1 = y;
    }
  }
}

template <int NC, class CT>
__device__ __forceinline__ void p1_from_xi(const CT (&t)[3], CT (&w)[NC]) {
  constexpr int D = NC == 4 ? 2 : 3;
  CT a0, a1, a2;
  int b0, b1, b2;
  p1_sorted<NC>(t, a0, a1, a2, b0, b1, b2);
  const int m1 = b0, m2 = b0 | b1;
  const CT v0 = CT(1) - a0, v1 = a0 - a1, v2 = D == 3 ? a1 - a2 : a1, v3 = a2;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    CT v = CT(0);
    if (c == 0) v = v0;
    else if (c == m1) v = v1;
    else if (c == m2) v = v2;
    else if (D == 3 && c == NC - 1) v = v3;
    w[c] = v;
  }
}

// the corners of the host box that are vertices of the Kuhn simplex holding t (bit c)
template <int NC, class CT>
__device__ __forceinline__ int p1_vertex_mask(const CT (&t)[3]) {
  CT a0, a1, a2;
  int b0, b1, b2;
  p1_sorted<NC>(t, a0, a1, a2, b0, b1, b2);
  return 1 | (1 << b0) | (1 << (b0 | b1)) | (1 << (NC - 1));
}

// Q1 values phi_c = prod_a (bit a of c ? xi_a : 1 - xi_a) at local coordinates
// t, multiplied in axis order (the same products as the stored Q1 values)
template <int NC, class CT>
__device__ __forceinline__ void q1_from_xi(const CT (&t)[3], CT (&w)[NC]) {
  const CT one = CT(1);
  const CT f0[2] = {one - t[0], t[0]}, f1[2] = {one - t[1], t[1]};
  if (NC == 4) {
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = f0[c & 1] * f1[(c >> 1) & 1];
  } else {
    const CT f2[2] = {one - t[2], t[2]};
    CT g[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) g[c] = f0[c & 1] * f1[c >> 1];
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = g[c & 3] * f2[(c >> 2) & 1];
  }
}

// the coarse basis values at local coordinates t: Q1, or P1 (simplex = 1)
template <int NC, class CT>
__device__ __forceinline__ void basis_from_xi(const CT (&t)[3], CT (&w)[NC], int simplex) {
  if (simplex) p1_from_xi<NC>(t, w);
  else q1_from_xi<NC>(t, w);
}

template <int N>
struct Pow2 {
  static constexpr int value = N <= 1 ? 1 : N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32;
};

// block sum of one value per thread into out[blockIdx.x]; fixed order
__device__ __forceinline__ void block_partial(double v, double* out, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    out[blockIdx.x] = t;
  }
  __syncthreads();
}

// true in the block that finishes last (its partials and everyone's are visible)
__device__ __forceinline__ bool last_block(unsigned* cnt) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// a thread's share of the sum of n partials: part[tid], part[tid + B], ... in
// that order, eight L2 loads in flight (the partials were written by other
// blocks or by the previous kernel)
__device__ __forceinline__ double thread_share(const double* part, int n) {
  double s = 0.0;
  constexpr int U = 8;
  for (int i0 = threadIdx.x; i0 < n; i0 += U * (int)blockDim.x) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      v[u] = i < n ? __ldcg(part + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) s += v[u];
  }
  return s;
}

// sum of n partials by one block in a fixed order (result valid in every thread)
__device__ __forceinline__ double block_sum(const double* part, int n, double* sh) {
  double s = thread_share(part, n);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();
  return t;
}

// three such sums at once (sh holds 3 * 32 doubles)
__device__ __forceinline__ void block_sum3(const double* p0, int n0, const double* p1, int n1, const double* p2,
                                           int n2, double* sh, double* out) {
  double s[3] = {thread_share(p0, n0), thread_share(p1, n1), thread_share(p2, n2)};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if ((threadIdx.x & 31) == 0) sh[32 * k + (threadIdx.x >> 5)] = s[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[32 * k + w];
    out[k] = t;
  }
  __syncthreads();
}

}  // namespace spnet
