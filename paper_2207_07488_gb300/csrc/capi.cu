// The C ABI (include/spnet.h): argument checks, handle life cycle, and the
// orchestration of set-up and solve.
#include <cmath>
#include <cstring>

#include "spnet_internal.cuh"

namespace spnet {
int assemble(int model, int64_t n_nodes, int64_t n_edges, const int64_t* edges, const double* coef,
             const double* dirs, int mem, cudaStream_t s, int64_t* row_ptr, int32_t* col,
             double* val, int64_t cap_nnz, int64_t* nnz_out);
int build_operator(int dim, int ndof, int64_t n_nodes, const double* coords, const int64_t* row_ptr,
                   const int32_t* col_idx, const double* vals, int64_t n_dir, const int64_t* dir,
                   const double* domain_hi, int mem, cudaStream_t s, spnet_op_s** out);
}  // namespace spnet

using namespace spnet;

static int setup_impl(spnet_op_s* op, double H, const int* gamma_faces, const spnet_options* opts,
                      spnet_pc_s** out) {
  if (!op) return fail(SPNET_ERR_BAD_INPUT, "setup_preconditioner: null operator");
  if (!(H > 0.0) || !std::isfinite(H)) return fail(SPNET_ERR_BAD_H, "setup_preconditioner: H must be > 0");
  spnet_options o{};
  o.precision = SPNET_PREC_MIXED;
  o.star_set = SPNET_STARS_INTERIOR;
  o.flexible = -1;
  o.max_restarts = 2;
  if (opts) o = *opts;
  if (o.precision != SPNET_PREC_FP64 && o.precision != SPNET_PREC_MIXED)
    return fail(SPNET_ERR_BAD_INPUT, "setup_preconditioner: unknown precision");
  if (o.star_set != SPNET_STARS_INTERIOR && o.star_set != SPNET_STARS_ALL)
    return fail(SPNET_ERR_BAD_INPUT, "setup_preconditioner: unknown star set");
  if (o.batch_rhs < 0 || o.batch_rhs > 32)
    return fail(SPNET_ERR_BAD_INPUT, "setup_preconditioner: batch_rhs must be in 0..32");
  if (o.star_map < 0 || o.star_map > 8)
    return fail(SPNET_ERR_BAD_INPUT, "setup_preconditioner: star_map must be in 0..8");
  if (o.patch != SPNET_PATCH_ELEMENT && o.patch != SPNET_PATCH_SUPPORT)
    return fail(SPNET_ERR_BAD_INPUT, "setup_preconditioner: unknown patch rule");
  if (o.coarse_space != SPNET_COARSE_Q1 && o.coarse_space != SPNET_COARSE_P1)
    return fail(SPNET_ERR_BAD_INPUT, "setup_preconditioner: unknown coarse space");
  spnet_pc_s* pc = new spnet_pc_s();
  pc->op = op;
  pc->mem.stream = op->stream;
  pc->precision = o.precision;
  pc->star_set = o.star_set;
  pc->flexible = o.flexible < 0 ? (o.precision == SPNET_PREC_MIXED ? 1 : 0) : (o.flexible ? 1 : 0);
  pc->max_restarts = o.max_restarts < 0 ? 0 : o.max_restarts;
  pc->batch_rhs = o.batch_rhs < 1 ? 1 : o.batch_rhs;
  pc->star_map = o.star_map;
  pc->patch = o.patch;
  pc->coarse_space = o.coarse_space;
  pc->panels = o.no_panels ? 0 : 1;
  pc->d = op->dim;
  pc->nc = 1 << op->dim;
  pc->ndof = op->ndof;
  pc->H = H;
  int64_t n_mesh = 1, n_elem = 1;
  for (int a = 0; a < 3; ++a) pc->nH[a] = 1;
  for (int a = 0; a < op->dim; ++a) {
    double q = op->domain[a] / H;
    long long n = llround(q);
    if (n < 1 || std::fabs(q - (double)n) > 1e-9 * q || n > (1 << 20)) {
      delete pc;
      return fail(SPNET_ERR_BAD_H, "setup_preconditioner: l_i / H is not an integer >= 1");
    }
    pc->nH[a] = (int)n;
    n_elem *= n;
    n_mesh *= (n + 1);
  }
  if (n_mesh > ((int64_t)1 << 30)) {
    delete pc;
    return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: mesh too fine");
  }
  pc->n_elem = (int)n_elem;
  pc->n_mesh = (int)n_mesh;
  for (int c = 0; c < op->ndof; ++c) pc->gamma[c] = gamma_faces ? gamma_faces[c] : 0;
  cudaStream_t s = op->stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  auto bail = [&](int rc) {
    cudaStreamSynchronize(s);
    pc->mem.free_all();
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    delete pc;
    return rc;
  };
  int rc;
  if ((rc = pc_setup_structure(pc))) return bail(rc);
  pc->G = 4 * num_sms();
  pc->PG = 16 * num_sms();
  pc->spmv_lanes = choose_spmv_lanes(pc->K);
  pc->spmv_blocks = spmv_grid(pc, pc->spmv_lanes);
  // coarse space: Galerkin matrix and its inverse
  if (pc->m0 > 0) {
    double* A0 = nullptr;
    const size_t bytes = sizeof(double) * (size_t)pc->m0 * pc->m0;
    if ((rc = pc->mem.alloc((void**)&A0, bytes))) return bail(rc);
    if ((rc = pc_galerkin(pc, A0))) return bail(rc);
    if ((rc = pc_coarse_invert(pc, A0))) return bail(rc);
    if ((rc = coarse_gemv_prepare(pc))) return bail(rc);
    if (pc->m0 <= A0_KEEP) pc->A0 = A0;
    else pc->mem.release(A0);
  }
  if ((rc = pc_factor_stars(pc))) return bail(rc);
  if ((rc = pc_elem_tables(pc))) return bail(rc);
  // work vectors
  const int64_t N = pc->N;
  if ((rc = pc->mem.get(&pc->x, N)) || (rc = pc->mem.get(&pc->r, N)) || (rc = pc->mem.get(&pc->r2, N)) || (rc = pc->mem.get(&pc->p, N)) ||
      (rc = pc->mem.get(&pc->q, N)) || (rc = pc->mem.get(&pc->z, N)) || (rc = pc->mem.get(&pc->b, N)) ||
      (rc = pc->mem.get(&pc->vtmp, N)) || (rc = pc->mem.alloc(&pc->w, (size_t)(pc->sum_s > 0 ? pc->sum_s : 1) * (pc->precision == SPNET_PREC_FP64 ? 8 : 4))) ||
      (rc = pc->mem.get(&pc->rc, pc->m0 > 0 ? pc->m0 : 1)) ||
      (rc = pc->mem.get(&pc->zc, pc->m0 > 0 ? pc->m0 : 1)) ||
      (rc = pc->mem.get(&pc->partial, 5 * pc->PG)) || (rc = pc->mem.get(&pc->pspmv, 64 * num_sms())) ||
      (rc = pc->mem.get(&pc->scal, 1)) ||
      (rc = pc->mem.get(&pc->epart, (size_t)pc->n_elem * pc->nc * pc->ndof)))
    return bail(rc);
  cudaMemsetAsync(pc->scal, 0, sizeof(Scal), s);
  if ((rc = spmv_lanes_tune(pc))) return bail(rc);
  if ((rc = star_map_tune(pc))) return bail(rc);
  if ((rc = batch_jw_tune(pc))) return bail(rc);
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) != cudaSuccess) return bail(fail(SPNET_ERR_CUDA, "setup_preconditioner: device error"));
  if (cudaGetLastError() != cudaSuccess) return bail(fail(SPNET_ERR_CUDA, "setup_preconditioner: launch error"));
  pc->setup_ms = elapsed_ms(e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  op->refcount++;
  *out = pc;
  return SPNET_OK;
}

extern "C" {

int spnet_assemble(int model, int64_t n_nodes, int64_t n_edges, const int64_t* edges,
                   const double* coef, const double* dirs, int mem, void* stream, int64_t* row_ptr,
                   int32_t* col, double* val, int64_t cap_nnz, int64_t* nnz_out) {
  cudaGetLastError();  // start from a clean error state
  if (!edges && n_edges > 0) return fail(SPNET_ERR_BAD_INPUT, "spnet_assemble: null edges");
  if (!row_ptr || !col || !val) return fail(SPNET_ERR_BAD_INPUT, "spnet_assemble: null output");
  return spnet::assemble(model, n_nodes, n_edges, edges, coef, dirs, mem, (cudaStream_t)stream,
                         row_ptr, col, val, cap_nnz, nnz_out);
}

int spnet_assemble_beam(int64_t n_nodes, int64_t n_edges, const int64_t* edges, const double* coords,
                        const double* coef, int64_t n_triples, const int64_t* triples, double EI, int mem,
                        void* stream, int64_t* row_ptr, int32_t* col, double* val, int64_t cap_nnz,
                        int64_t* nnz_out) {
  cudaGetLastError();
  if ((!edges || !coef) && n_edges > 0) return fail(SPNET_ERR_BAD_INPUT, "spnet_assemble_beam: null edges");
  if (!coords || (!triples && n_triples > 0)) return fail(SPNET_ERR_BAD_INPUT, "spnet_assemble_beam: null input");
  if (!row_ptr || !col || !val) return fail(SPNET_ERR_BAD_INPUT, "spnet_assemble_beam: null output");
  return spnet::assemble_beam(n_nodes, n_edges, edges, coords, coef, n_triples, triples, EI, mem,
                              (cudaStream_t)stream, row_ptr, col, val, cap_nnz, nnz_out);
}

int build_network_operator(int dim, int ndof, int64_t n_nodes, const double* coords,
                           const int64_t* row_ptr, const int32_t* col_idx, const double* vals,
                           int64_t n_dirichlet, const int64_t* dirichlet_dofs,
                           const double* domain_hi, int mem, void* stream, spnet_op_t* out) {
  cudaGetLastError();  // start from a clean error state
  if (!out || !coords || !row_ptr || !col_idx || !vals || !domain_hi || (n_dirichlet > 0 && !dirichlet_dofs))
    return fail(SPNET_ERR_BAD_INPUT, "build_network_operator: null argument");
  if (mem != SPNET_MEM_HOST && mem != SPNET_MEM_DEVICE)
    return fail(SPNET_ERR_BAD_INPUT, "build_network_operator: bad mem flag");
  spnet_op_s* op = nullptr;
  int rc = spnet::build_operator(dim, ndof, n_nodes, coords, row_ptr, col_idx, vals, n_dirichlet,
                                 dirichlet_dofs, domain_hi, mem, (cudaStream_t)stream, &op);
  if (rc == SPNET_OK) *out = op;
  return rc;
}

int setup_preconditioner(spnet_op_t op, double H, const int* gamma_faces, const spnet_options* opts,
                         spnet_pc_t* out) {
  cudaGetLastError();  // start from a clean error state
  if (!out) return fail(SPNET_ERR_BAD_INPUT, "setup_preconditioner: null output");
  spnet_pc_s* pc = nullptr;
  int rc = setup_impl(op, H, gamma_faces, opts, &pc);
  if (rc == SPNET_OK) *out = pc;
  return rc;
}

int pcg_solve(spnet_op_t op, spnet_pc_t pc, int nrhs, const double* f, const double* g, double* x,
              int use_x0, double rtol, int maxit, int mem, spnet_stats* stats) {
  cudaGetLastError();  // start from a clean error state
  if (!op || !pc || pc->op != op) return fail(SPNET_ERR_BAD_INPUT, "pcg_solve: operator/preconditioner mismatch");
  if (nrhs < 0 || !f || !x || (op->n_dir > 0 && !g)) return fail(SPNET_ERR_BAD_INPUT, "pcg_solve: null argument");
  if (!(rtol > 0.0) || maxit < 0) return fail(SPNET_ERR_BAD_INPUT, "pcg_solve: rtol must be > 0, maxit >= 0");
  if (mem != SPNET_MEM_HOST && mem != SPNET_MEM_DEVICE) return fail(SPNET_ERR_BAD_INPUT, "pcg_solve: bad mem flag");
  if (nrhs == 0) return SPNET_OK;
  return spnet::pcg_run(op, pc, nrhs, f, g, x, use_x0, rtol, maxit, mem, stats);
}

int spnet_op_destroy(spnet_op_t op) {
  cudaGetLastError();  // start from a clean error state
  if (!op) return SPNET_OK;
  if (op->refcount > 0) return fail(SPNET_ERR_BAD_INPUT, "spnet_op_destroy: preconditioners still alive");
  cudaStream_t s = op->stream;
  op->mem.free_all();
  cudaStreamSynchronize(s);
  if (op->own_stream) cudaStreamDestroy(s);
  delete op;
  return SPNET_OK;
}

int spnet_pc_destroy(spnet_pc_t pc) {
  cudaGetLastError();  // start from a clean error state
  if (!pc) return SPNET_OK;
  cudaStream_t s = pc->op->stream;
  cudaStreamSynchronize(s);
  if (pc->graph_exec) cudaGraphExecDestroy(pc->graph_exec);
  if (pc->side) {
    cudaStreamSynchronize(pc->side);
    cudaStreamDestroy(pc->side);
  }
  if (pc->ev_fork) cudaEventDestroy(pc->ev_fork);
  if (pc->ev_join) cudaEventDestroy(pc->ev_join);
  pc->mem.free_all();
  cudaStreamSynchronize(s);
  pc->op->refcount--;
  delete pc;
  return SPNET_OK;
}

int spnet_last_error(char* buf, size_t len) {
  if (!buf || len == 0) return SPNET_ERR_BAD_INPUT;
  const std::string& m = last_error();
  size_t n = m.size() < len - 1 ? m.size() : len - 1;
  std::memcpy(buf, m.data(), n);
  buf[n] = 0;
  return SPNET_OK;
}

int spnet_op_get_info(spnet_op_t op, spnet_op_info* info) {
  cudaGetLastError();  // start from a clean error state
  if (!op || !info) return fail(SPNET_ERR_BAD_INPUT, "spnet_op_get_info: null argument");
  *info = spnet_op_info{};
  info->n_dof = op->n_dof;
  info->n_free = op->n_free;
  info->n_dirichlet = op->n_dir;
  info->nnz_ff = op->ff.nnz;
  info->nnz_fd = op->fd.nnz;
  info->dim = op->dim;
  info->ndof = op->ndof;
  return SPNET_OK;
}

int spnet_pc_get_info(spnet_pc_t pc, spnet_pc_info* info) {
  cudaGetLastError();  // start from a clean error state
  if (!pc || !info) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_get_info: null argument");
  *info = spnet_pc_info{};
  for (int a = 0; a < 3; ++a) info->nH[a] = pc->nH[a];
  info->n_elem = pc->n_elem;
  info->n_mesh = pc->n_mesh;
  info->m0 = pc->m0;
  info->n_stars = pc->S;
  info->max_star = pc->max_star;
  info->sum_star = pc->sum_s;
  info->factor_nnz = pc->factor_nnz;
  info->total_levels = pc->total_levels;
  info->max_levels = pc->max_levels;
  info->precision = pc->precision;
  info->star_set = pc->star_set;
  info->flexible = pc->flexible;
  info->setup_ms = pc->setup_ms;
  info->device_bytes = pc->mem.bytes;
  info->star_stream_bytes = pc->stream_bytes;
  info->star_warps_per_block = pc->solve_wpb;
  info->coarse_dropped = pc->coarse_dropped;
  info->panel_stars = pc->panel_stars;
  info->tuned = pc->spmv_lanes + 256ll * pc->batch_jw;
  return SPNET_OK;
}

static int with_free_vectors(spnet_pc_s* pc, const double* in, int64_t nin, double* out, int64_t nout,
                             int mem, int (*fn)(spnet_pc_s*, const double*, double*)) {
  cudaStream_t s = pc->op->stream;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const double* din = in;
  double* dout = out;
  if (mem == SPNET_MEM_HOST) {
    double *a = nullptr, *b = nullptr;
    SPNET_TRY(tmp.get(&a, nin > 0 ? nin : 1));
    SPNET_TRY(tmp.get(&b, nout > 0 ? nout : 1));
    SPNET_TRY(copy_in(in, a, sizeof(double) * nin, mem, s));
    din = a;
    dout = b;
  }
  SPNET_TRY(fn(pc, din, dout));
  if (mem == SPNET_MEM_HOST) SPNET_TRY(copy_out(dout, out, sizeof(double) * nout, mem, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  SPNET_CUDA_TRY(cudaGetLastError());
  return SPNET_OK;
}

int spnet_spmv(spnet_op_t op, const double* x, double* y, int mem) {
  cudaGetLastError();  // start from a clean error state
  if (!op || !x || !y) return fail(SPNET_ERR_BAD_INPUT, "spnet_spmv: null argument");
  cudaStream_t s = op->stream;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const double* dx = x;
  double* dy = y;
  if (mem == SPNET_MEM_HOST) {
    double *a = nullptr, *b = nullptr;
    SPNET_TRY(tmp.get(&a, op->n_free));
    SPNET_TRY(tmp.get(&b, op->n_free));
    SPNET_TRY(copy_in(x, a, sizeof(double) * op->n_free, mem, s));
    dx = a;
    dy = b;
  }
  launch_spmv(op->ff, dx, dy, nullptr, 4 * num_sms(), choose_spmv_lanes(op->ff), nullptr, s);
  if (mem == SPNET_MEM_HOST) SPNET_TRY(copy_out(dy, y, sizeof(double) * op->n_free, mem, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  SPNET_CUDA_TRY(cudaGetLastError());
  return SPNET_OK;
}

static int apply_all(spnet_pc_s* pc, const double* r, double* z) { return pc_apply_free(pc, r, z, 0); }
static int apply_star_term(spnet_pc_s* pc, const double* r, double* z) { return pc_apply_free(pc, r, z, 2); }

int spnet_pc_apply(spnet_pc_t pc, const double* r, double* z, int mem) {
  cudaGetLastError();  // start from a clean error state
  if (!pc || !r || !z) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_apply: null argument");
  return with_free_vectors(pc, r, pc->N, z, pc->N, mem, apply_all);
}

int spnet_pc_apply_batch(spnet_pc_t pc, int k, const double* r, double* z, int which, int mem) {
  cudaGetLastError();  // start from a clean error state
  if (!pc || !r || !z) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_apply_batch: null argument");
  if (k < 1 || k > 32) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_apply_batch: k must be in 1..32");
  if (which < 0 || which > 2) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_apply_batch: which must be 0, 1 or 2");
  if (mem != SPNET_MEM_HOST && mem != SPNET_MEM_DEVICE)
    return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_apply_batch: bad mem flag");
  cudaStream_t s = pc->op->stream;
  const int64_t n = (int64_t)k * pc->N;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const double* din = r;
  double* dout = z;
  if (mem == SPNET_MEM_HOST) {
    double *a = nullptr, *b = nullptr;
    SPNET_TRY(tmp.get(&a, n > 0 ? n : 1));
    SPNET_TRY(tmp.get(&b, n > 0 ? n : 1));
    SPNET_TRY(copy_in(r, a, sizeof(double) * n, mem, s));
    din = a;
    dout = b;
  }
  // passes of at most the block width whose star solve fits a block's shared memory
  const int kmax = star_batch_max_k(pc);
  for (int k0 = 0; k0 < k; k0 += kmax) {
    const int kk = k - k0 < kmax ? k - k0 : kmax;
    SPNET_TRY(pc_apply_batch_free(pc, kk, din + (int64_t)k0 * pc->N, dout + (int64_t)k0 * pc->N, which));
  }
  if (mem == SPNET_MEM_HOST) SPNET_TRY(copy_out(dout, z, sizeof(double) * n, mem, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  SPNET_CUDA_TRY(cudaGetLastError());
  return SPNET_OK;
}

int spnet_pc_stars(spnet_pc_t pc, const double* r, double* z, int mem) {
  cudaGetLastError();  // start from a clean error state
  if (!pc || !r || !z) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_stars: null argument");
  return with_free_vectors(pc, r, pc->N, z, pc->N, mem, apply_star_term);
}

static int restrict_fn(spnet_pc_s* pc, const double* r, double* rc) {
  return pc_restrict_free(pc, r, rc);
}

static int coarse_fn(spnet_pc_s* pc, const double* rc, double* zc) {
  launch_coarse_apply(pc, rc, zc, nullptr, pc->op->stream);
  return SPNET_OK;
}

static int prolong_fn(spnet_pc_s* pc, const double* zc, double* z) {
  cudaStream_t s = pc->op->stream;
  if (pc->m0 > 0)
    SPNET_CUDA_TRY(cudaMemcpyAsync(pc->zc, zc, sizeof(double) * pc->m0, cudaMemcpyDeviceToDevice, s));
  launch_combine(pc, pc->vtmp, pc->z, 1, 0, 0, s, 1);  // the stand-alone prolongation: FP64
  from_pc(pc, pc->z, z);
  return SPNET_OK;
}

int spnet_pc_restrict(spnet_pc_t pc, const double* r, double* rc, int mem) {
  cudaGetLastError();  // start from a clean error state
  if (!pc || !r || !rc) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_restrict: null argument");
  return with_free_vectors(pc, r, pc->N, rc, pc->m0, mem, restrict_fn);
}

int spnet_pc_coarse(spnet_pc_t pc, const double* rc, double* zc, int mem) {
  cudaGetLastError();  // start from a clean error state
  if (!pc || !rc || !zc) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_coarse: null argument");
  return with_free_vectors(pc, rc, pc->m0, zc, pc->m0, mem, coarse_fn);
}

int spnet_pc_prolong(spnet_pc_t pc, const double* zc, double* z, int mem) {
  cudaGetLastError();  // start from a clean error state
  if (!pc || !zc || !z) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_prolong: null argument");
  return with_free_vectors(pc, zc, pc->m0, z, pc->N, mem, prolong_fn);
}

int spnet_pc_export(spnet_pc_t pc, int what, void* host_buf, size_t bytes) {
  cudaGetLastError();  // start from a clean error state
  if (!pc || !host_buf) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_export: null argument");
  cudaStream_t s = pc->op->stream;
  size_t need = 0;
  switch (what) {
    case SPNET_EXPORT_ELEMENTS: need = sizeof(int32_t) * pc->N; break;
    case SPNET_EXPORT_Q1: need = sizeof(double) * pc->N * pc->nc; break;
    case SPNET_EXPORT_COARSE_MAP: need = sizeof(int32_t) * (size_t)pc->n_mesh * pc->ndof; break;
    case SPNET_EXPORT_STAR_SIZES: case SPNET_EXPORT_STAR_MESH: case SPNET_EXPORT_STAR_LEVELS:
    case SPNET_EXPORT_STAR_CORE:
      need = sizeof(int32_t) * pc->S; break;
    case SPNET_EXPORT_A0:
      if (!pc->A0 && pc->m0 > 0) return fail(SPNET_ERR_UNSUPPORTED, "spnet_pc_export: A_0 is kept only for m0 <= 2048");
      need = sizeof(double) * (size_t)pc->m0 * pc->m0; break;
    default: return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_export: unknown item");
  }
  if (bytes < need) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_export: buffer too small");
  int rc = export_item(pc, what, host_buf);
  if (rc) return rc;
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  return SPNET_OK;
}

int spnet_launch_count(int64_t* count) {
  cudaGetLastError();  // start from a clean error state
  if (!count) return fail(SPNET_ERR_BAD_INPUT, "spnet_launch_count: null argument");
  *count = (int64_t)launch_count();
  return SPNET_OK;
}

int spnet_profile_enable(int on) {
  cudaGetLastError();  // start from a clean error state
  profile_enable(on);
  return SPNET_OK;
}

int spnet_profile_read(int kernel, int64_t* launches, double* total_ms) {
  cudaGetLastError();  // start from a clean error state
  if (kernel < 0 || kernel >= KID_COUNT || !launches || !total_ms)
    return fail(SPNET_ERR_BAD_INPUT, "spnet_profile_read: bad argument");
  long long n = 0;
  double ms = 0.0;
  profile_read(kernel, &n, &ms);
  *launches = n;
  *total_ms = ms;
  return SPNET_OK;
}

int spnet_profile_reset(void) {
  cudaGetLastError();  // start from a clean error state
  profile_reset();
  return SPNET_OK;
}

int spnet_pc_record_iterates(spnet_pc_t pc, double* buf, int64_t max_iterates) {
  cudaGetLastError();  // start from a clean error state
  if (!pc) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_record_iterates: null preconditioner");
  if (max_iterates < 0 || (buf == nullptr) != (max_iterates == 0))
    return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_record_iterates: buf and max_iterates disagree");
  if (buf) {
    if (reinterpret_cast<uintptr_t>(buf) % 8 != 0)
      return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_record_iterates: buf not 8-byte aligned");
    if (pc->N > 0 && max_iterates > (((int64_t)1 << 62) / pc->N))
      return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_record_iterates: max_iterates * n_free beyond 2^62");
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, buf);
    if (e != cudaSuccess) cudaGetLastError();
    if (e != cudaSuccess || (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) ||
        a.device != pc->op->device)
      return fail(SPNET_ERR_BAD_INPUT,
                  "spnet_pc_record_iterates: buf is not device memory of the preconditioner's device");
  }
  pc->rec_buf = buf;
  pc->rec_max = max_iterates;
  return SPNET_OK;
}

}  // extern "C"
