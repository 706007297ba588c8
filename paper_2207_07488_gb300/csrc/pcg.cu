// Preconditioned conjugate gradients (Section 4.2) on the free dofs in pc
// order, and the restriction / combination steps of B (Section 4.1).
//
// Each iteration is a fixed sequence of kernels:
//   spmv      q = A p, partial (p, q)
//   update    alpha = (r, z)/(p, q); x += alpha p; r -= alpha q; partial |r|^2
//   restrict  stop test |r| <= rtol |b| (sets `done`), r_c = R_0 r
//   stars     w_j = A_j^{-1} E_j^T r for every star
//   coarse    z_c = A_0^{-1} r_c
//   combine   z = R_0^T z_c + sum_j E_j w_j, partial (r, z) [and (r, z_old)]
//   direction beta; p = z + beta p
// Every kernel returns at once when `done` is set, so the host may launch
// several iterations ahead and read the state only now and then.  Partial
// sums use a fixed grid and are reduced in a fixed order by every block:
// results are bitwise reproducible.  Scalars live on the device; a value a
// kernel publishes is read only by later kernels.
#include <cmath>

#include "spnet_internal.cuh"

namespace spnet {

__device__ __forceinline__ double block_reduce_partials(const double* partial, int G, double* sh) {
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < G; i += 32) s += partial[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) sh[0] = s;
  }
  __syncthreads();
  double v = sh[0];
  __syncthreads();
  return v;
}

__device__ __forceinline__ void block_write_partial(double v, double* out, double* sh) {
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

#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// b = f_I - K_ID g (Section 3), in pc order
__global__ void k_build_rhs(int64_t N, const int32_t* perm, const int64_t* free_dofs, const double* f,
                            const int64_t* fdp, const int32_t* fdc, const double* fdv, const double* g,
                            double* b) {
  GRID_STRIDE(p, N) {
    int32_t fi = perm[p];
    double s = f[free_dofs[fi]];
    for (int64_t k = fdp[fi]; k < fdp[fi + 1]; ++k) s -= fdv[k] * g[fdc[k]];
    b[p] = s;
  }
}

__global__ void k_to_pc(int64_t N, const int32_t* perm, const double* xf, double* xp) {
  GRID_STRIDE(p, N) xp[p] = xf[perm[p]];
}

__global__ void k_from_pc(int64_t N, const int32_t* perm, const double* xp, double* xf) {
  GRID_STRIDE(p, N) xf[perm[p]] = xp[p];
}

__global__ void k_x0_from_dofs(int64_t N, const int32_t* perm, const int64_t* free_dofs, const double* x,
                               double* xp) {
  GRID_STRIDE(p, N) xp[p] = x[free_dofs[perm[p]]];
}

// u_hat on all dofs: x at free dofs, g at Dirichlet dofs
__global__ void k_expand(int64_t n_dof, const int64_t* free_of, const int32_t* iperm, const double* xp,
                         const double* g, double* out) {
  GRID_STRIDE(v, n_dof) {
    int64_t f = free_of[v];
    out[v] = f >= 0 ? xp[iperm[f]] : g[-f - 2];
  }
}

__global__ void k_dot_partial(int64_t N, const double* a, const double* b, double* partial) {
  __shared__ double sh[32];
  double s = 0.0;
  GRID_STRIDE(i, N) s = fma(a[i], b[i], s);
  block_write_partial(s, partial, sh);
}

__global__ void k_reduce_to(const double* partial, int G, double* out) {
  __shared__ double sh[1];
  double v = block_reduce_partials(partial, G, sh);
  if (threadIdx.x == 0) *out = v;
}

// r = b - q, partial |r|^2
__global__ void k_residual(int64_t N, const double* b, const double* q, double* r, double* partial) {
  __shared__ double sh[32];
  double s = 0.0;
  GRID_STRIDE(i, N) {
    double v = b[i] - q[i];
    r[i] = v;
    s = fma(v, v, s);
  }
  block_write_partial(s, partial, sh);
}

__global__ void k_update_xr(int64_t N, double* x, double* r, const double* p, const double* q,
                            const double* part_pq, double* part_rr, int G, Scal* sc) {
  __shared__ double sh[32];
  if (sc->done) return;
  const double pq = block_reduce_partials(part_pq, G, sh);
  const double rz = sc->rz_old;  // (r, z) published by the previous direction update
  const double alpha = rz / pq;
  double s = 0.0;
  GRID_STRIDE(i, N) {
    x[i] = fma(alpha, p[i], x[i]);
    double v = fma(-alpha, q[i], r[i]);
    r[i] = v;
    s = fma(v, v, s);
  }
  block_write_partial(s, part_rr, sh);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->pq = pq;
    sc->alpha = alpha;
    sc->rz = rz;
    sc->iter += 1;
  }
}

// r_c = R_0 r; one warp per mesh node; optionally the stop test first
__global__ void k_restrict(int n_mesh, Mesh m, int ndof, int64_t N, const int32_t* elem_ptr,
                           const int8_t* comp_of, const double* q1w, const int32_t* cidx,
                           const double* r, double* rc, Scal* sc, const double* part_rr, int G,
                           double tol2_rel, int maxit) {
  __shared__ double sh[1];
  if (sc) {
    if (sc->done) return;
    const double rr = block_reduce_partials(part_rr, G, sh);
    const bool stop = sqrt(rr) <= tol2_rel * sqrt(sc->bb) || sc->iter >= maxit;
    if (stop) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->rr = rr;
        sc->done = 1;
      }
      return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->rr = rr;
  }
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_mesh; k += nw) {
    bool any = false;
    for (int a = 0; a < ndof; ++a) any |= cidx[k * ndof + a] >= 0;
    if (!any) continue;
    int km[3];
    mesh_multi(m, (int)k, km);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int cp = 0; cp < m.nc; ++cp) {
      int e = elem_around(m, km, cp);
      if (e < 0) continue;
      const int c = (m.nc - 1) - cp;  // corner of e at mesh node k
      const double* wc = q1w + (int64_t)c * N;
      for (int p = elem_ptr[e] + lane; p < elem_ptr[e + 1]; p += 32) {
        double v = wc[p] * r[p];
        if (ndof == 1) acc[0] += v;
        else acc[comp_of[p]] += v;
      }
    }
    for (int a = 0; a < ndof; ++a) {
      double v = acc[a];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      int ci = cidx[k * ndof + a];
      if (lane == 0 && ci >= 0) rc[ci] = v;
    }
  }
}

// z = [R_0^T z_c] + [sum_j E_j w_j]; partial (r, z) and (r, z_old)
__global__ void k_combine(int64_t N, Mesh m, int ndof, const int32_t* elem_of, const int8_t* comp_of,
                          const int32_t* elem_ptr, const double* q1w, const int32_t* cidx,
                          const double* zc, const int32_t* elem_star_off, const int32_t* star_of_mesh,
                          const int64_t* star_ptr, const double* w, const double* r, double* z,
                          double* part_rz, double* part_rzo, int with_coarse, int with_stars,
                          const int* done) {
  __shared__ double sh[32];
  if (done && *done) return;
  double s1 = 0.0, s2 = 0.0;
  GRID_STRIDE(p, N) {
    const int e = elem_of[p];
    const int a = ndof == 1 ? 0 : comp_of[p];
    double v = 0.0;
    if (with_coarse) {
      for (int c = 0; c < m.nc; ++c) {
        int ci = cidx[(int64_t)mesh_of(m, e, c) * ndof + a];
        if (ci >= 0) v = fma(q1w[(int64_t)c * N + p], zc[ci], v);
      }
    }
    if (with_stars) {
      const int off_e = (int)(p - elem_ptr[e]);
      for (int c = 0; c < m.nc; ++c) {
        int so = elem_star_off[(int64_t)e * m.nc + c];
        if (so < 0) continue;
        int st = star_of_mesh[mesh_of(m, e, c)];
        v += w[star_ptr[st] + so + off_e];
      }
    }
    if (part_rz) {
      s1 = fma(r[p], v, s1);
      if (part_rzo) s2 = fma(r[p], z[p], s2);
    }
    z[p] = v;
  }
  if (part_rz) {
    block_write_partial(s1, part_rz, sh);
    if (part_rzo) block_write_partial(s2, part_rzo, sh);
  }
}

// beta and p = z + beta p
__global__ void k_direction(int64_t N, const double* z, double* p, const double* part_rz,
                            const double* part_rzo, int G, int flexible, int first, Scal* sc) {
  __shared__ double sh[1];
  if (sc->done) return;
  const double rz_new = block_reduce_partials(part_rz, G, sh);
  double beta = 0.0;
  if (!first) {
    const double rz = sc->rz;
    if (flexible) {
      const double rzo = block_reduce_partials(part_rzo, G, sh);
      beta = (rz_new - rzo) / rz;
    } else {
      beta = rz_new / rz;
    }
  }
  GRID_STRIDE(i, N) p[i] = first ? z[i] : fma(beta, p[i], z[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->beta = beta;
    sc->rz_old = rz_new;
  }
}

__global__ void k_copy(int64_t N, const double* a, double* b) {
  GRID_STRIDE(i, N) b[i] = a[i];
}

void launch_restrict(spnet_pc_s* pc, const double* r, double* rc, const int* done, cudaStream_t s) {
  (void)done;
  if (pc->m0 == 0) return;
  int blocks = (pc->n_mesh + 7) / 8;
  note_launch();
  k_restrict<<<blocks, 256, 0, s>>>(pc->n_mesh, mesh_of_pc(pc), pc->ndof, pc->N, pc->elem_ptr,
                                    pc->comp_of, pc->q1w, pc->cidx, r, rc, nullptr, nullptr, 0, 0.0, 0);
}

void launch_combine(spnet_pc_s* pc, const double* r, double* z, int with_coarse, int with_stars,
                    int with_dots, const int* done, cudaStream_t s) {
  double* prz = with_dots ? pc->partial + 2 * pc->G : nullptr;
  double* przo = (with_dots && pc->flexible) ? pc->partial + 3 * pc->G : nullptr;
  note_launch();
  ProfScope ps(KID_COMBINE, s);
  k_combine<<<pc->G, RED_BLOCK, 0, s>>>(pc->N, mesh_of_pc(pc), pc->ndof, pc->elem_of, pc->comp_of,
                                        pc->elem_ptr, pc->q1w, pc->cidx, pc->zc, pc->elem_star_off,
                                        pc->star_of_mesh, pc->star_ptr, pc->w, r, z, prz, przo,
                                        with_coarse && pc->m0 > 0, with_stars && pc->S > 0, done);
}

// z = B r (pc order), without the stop test
static void precond(spnet_pc_s* pc, const double* r, double* z, int with_dots, const int* done,
                    cudaStream_t s) {
  if (pc->m0 > 0) {
    launch_restrict(pc, r, pc->rc, done, s);
    launch_coarse_apply(pc, pc->rc, pc->zc, done, s);
  }
  launch_star_solve(pc, r, done, s);
  launch_combine(pc, r, z, 1, 1, with_dots, done, s);
}

// one PCG iteration (see the file comment)
static void iteration(spnet_pc_s* pc, double rtol, int maxit, cudaStream_t s) {
  const int G = pc->G;
  int* done = &pc->scal->done;
  launch_spmv(pc->K, pc->p, pc->q, pc->partial, G, pc->spmv_lanes, done, s);
  note_launch();
  {
  ProfScope ps(KID_UPDATE, s);
  k_update_xr<<<G, RED_BLOCK, 0, s>>>(pc->N, pc->x, pc->r, pc->p, pc->q, pc->partial,
                                      pc->partial + G, G, pc->scal);
  }
  {
    ProfScope ps(KID_RESTRICT, s);
    int blocks = pc->m0 > 0 ? (pc->n_mesh + 7) / 8 : 1;
    note_launch();
    k_restrict<<<blocks, 256, 0, s>>>(pc->m0 > 0 ? pc->n_mesh : 0, mesh_of_pc(pc), pc->ndof, pc->N,
                                      pc->elem_ptr, pc->comp_of, pc->q1w, pc->cidx, pc->r, pc->rc,
                                      pc->scal, pc->partial + G, G, rtol, maxit);
  }
  if (pc->m0 > 0) launch_coarse_apply(pc, pc->rc, pc->zc, done, s);
  launch_star_solve(pc, pc->r, done, s);
  launch_combine(pc, pc->r, pc->z, 1, 1, 1, done, s);
  note_launch();
  ProfScope ps(KID_DIRECTION, s);
  k_direction<<<G, RED_BLOCK, 0, s>>>(pc->N, pc->z, pc->p, pc->partial + 2 * G, pc->partial + 3 * G,
                                      G, pc->flexible, 0, pc->scal);
}

void to_pc(spnet_pc_s* pc, const double* free_vec, double* pc_vec) {
  note_launch();
  k_to_pc<<<pc->G, 256, 0, pc->op->stream>>>(pc->N, pc->perm, free_vec, pc_vec);
}

void from_pc(spnet_pc_s* pc, const double* pc_vec, double* free_vec) {
  note_launch();
  k_from_pc<<<pc->G, 256, 0, pc->op->stream>>>(pc->N, pc->perm, pc_vec, free_vec);
}

__global__ void k_export_elem(int64_t N, const int32_t* iperm, const int32_t* elem_of, int32_t* out) {
  GRID_STRIDE(f, N) out[f] = elem_of[iperm[f]];
}

__global__ void k_export_q1(int64_t N, int nc, const int32_t* iperm, const double* q1w, double* out) {
  GRID_STRIDE(f, N) {
    for (int c = 0; c < nc; ++c) out[f * nc + c] = q1w[(int64_t)c * N + iperm[f]];
  }
}

int export_item(spnet_pc_s* pc, int what, void* host_buf) {
  cudaStream_t s = pc->op->stream;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  switch (what) {
    case SPNET_EXPORT_ELEMENTS: {
      int32_t* d = nullptr;
      SPNET_TRY(tmp.get(&d, pc->N));
      note_launch();
      k_export_elem<<<pc->G, 256, 0, s>>>(pc->N, pc->iperm, pc->elem_of, d);
      SPNET_CUDA_TRY(cudaMemcpyAsync(host_buf, d, sizeof(int32_t) * pc->N, cudaMemcpyDeviceToHost, s));
      break;
    }
    case SPNET_EXPORT_Q1: {
      double* d = nullptr;
      SPNET_TRY(tmp.get(&d, pc->N * pc->nc));
      note_launch();
      k_export_q1<<<pc->G, 256, 0, s>>>(pc->N, pc->nc, pc->iperm, pc->q1w, d);
      SPNET_CUDA_TRY(cudaMemcpyAsync(host_buf, d, sizeof(double) * pc->N * pc->nc, cudaMemcpyDeviceToHost, s));
      break;
    }
    case SPNET_EXPORT_COARSE_MAP:
      SPNET_CUDA_TRY(cudaMemcpyAsync(host_buf, pc->cidx, sizeof(int32_t) * (size_t)pc->n_mesh * pc->ndof,
                                     cudaMemcpyDeviceToHost, s));
      break;
    case SPNET_EXPORT_STAR_SIZES:
      if (pc->S) SPNET_CUDA_TRY(cudaMemcpyAsync(host_buf, pc->star_n, sizeof(int32_t) * pc->S, cudaMemcpyDeviceToHost, s));
      break;
    case SPNET_EXPORT_STAR_MESH:
      if (pc->S) SPNET_CUDA_TRY(cudaMemcpyAsync(host_buf, pc->star_mesh, sizeof(int32_t) * pc->S, cudaMemcpyDeviceToHost, s));
      break;
    case SPNET_EXPORT_STAR_LEVELS:
      if (pc->S) SPNET_CUDA_TRY(cudaMemcpyAsync(host_buf, pc->star_lev, sizeof(int32_t) * pc->S, cudaMemcpyDeviceToHost, s));
      break;
    case SPNET_EXPORT_A0:
      if (pc->m0) SPNET_CUDA_TRY(cudaMemcpyAsync(host_buf, pc->A0, sizeof(double) * (size_t)pc->m0 * pc->m0,
                                                 cudaMemcpyDeviceToHost, s));
      break;
    default:
      return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_export: unknown item");
  }
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  return SPNET_OK;
}

int pc_apply_free(spnet_pc_s* pc, const double* r_free, double* z_free, int which) {
  cudaStream_t s = pc->op->stream;
  const int grid = pc->G;
  note_launch();
  k_to_pc<<<grid, 256, 0, s>>>(pc->N, pc->perm, r_free, pc->vtmp);
  if (which == 0) {
    precond(pc, pc->vtmp, pc->z, 0, nullptr, s);
  } else if (which == 1) {  // coarse term only
    if (pc->m0 > 0) {
      launch_restrict(pc, pc->vtmp, pc->rc, nullptr, s);
      launch_coarse_apply(pc, pc->rc, pc->zc, nullptr, s);
    }
    launch_combine(pc, pc->vtmp, pc->z, 1, 0, 0, nullptr, s);
  } else {  // star term only
    launch_star_solve(pc, pc->vtmp, nullptr, s);
    launch_combine(pc, pc->vtmp, pc->z, 0, 1, 0, nullptr, s);
  }
  note_launch();
  k_from_pc<<<grid, 256, 0, s>>>(pc->N, pc->perm, pc->z, z_free);
  SPNET_CUDA_TRY(cudaGetLastError());
  return SPNET_OK;
}

int pcg_run(spnet_op_s* op, spnet_pc_s* pc, int nrhs, const double* f, const double* g, double* x,
            int use_x0, double rtol, int maxit, int mem, spnet_stats* stats) {
  cudaStream_t s = op->stream;
  const int64_t N = pc->N, nd = op->n_dof, ndir = op->n_dir;
  const int G = pc->G;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const double *df = f, *dg = g;
  double* dx = x;
  if (mem == SPNET_MEM_HOST) {
    double *a = nullptr, *b = nullptr, *c = nullptr;
    SPNET_TRY(tmp.get(&a, (size_t)nrhs * nd));
    SPNET_TRY(tmp.get(&b, (size_t)nrhs * (ndir > 0 ? ndir : 1)));
    SPNET_TRY(tmp.get(&c, (size_t)nrhs * nd));
    SPNET_TRY(copy_in(f, a, sizeof(double) * nrhs * nd, mem, s));
    SPNET_TRY(copy_in(g, b, sizeof(double) * nrhs * ndir, mem, s));
    if (use_x0) SPNET_TRY(copy_in(x, c, sizeof(double) * nrhs * nd, mem, s));
    df = a;
    dg = b;
    dx = c;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int worst = SPNET_OK;
  const int chunk = 8;
  for (int k = 0; k < nrhs; ++k) {
    const double* fk = df + (int64_t)k * nd;
    const double* gk = dg + (int64_t)k * ndir;
    double* xk = dx + (int64_t)k * nd;
    cudaEventRecord(e0, s);
    SPNET_CUDA_TRY(cudaMemsetAsync(pc->scal, 0, sizeof(Scal), s));
    note_launch();
    k_build_rhs<<<G, 256, 0, s>>>(N, pc->perm, op->free_dofs, fk, op->fd.ptr, op->fd.col, op->fd.val,
                                  gk, pc->b);
    note_launch();
    k_dot_partial<<<G, RED_BLOCK, 0, s>>>(N, pc->b, pc->b, pc->partial);
    note_launch();
    k_reduce_to<<<1, 32, 0, s>>>(pc->partial, G, &pc->scal->bb);
    if (use_x0) {
      note_launch();
      k_x0_from_dofs<<<G, 256, 0, s>>>(N, pc->perm, op->free_dofs, xk, pc->x);
      launch_spmv(pc->K, pc->x, pc->q, nullptr, G, pc->spmv_lanes, nullptr, s);
    } else {
      SPNET_CUDA_TRY(cudaMemsetAsync(pc->x, 0, sizeof(double) * N, s));
      SPNET_CUDA_TRY(cudaMemsetAsync(pc->q, 0, sizeof(double) * N, s));
    }
    int restarts = 0;
    Scal h{};
    for (;;) {
      // (re)start: r = b - A x, z = B r, p = z
      note_launch();
      k_residual<<<G, RED_BLOCK, 0, s>>>(N, pc->b, pc->q, pc->r, pc->partial + G);
      note_launch();
      k_reduce_to<<<1, 32, 0, s>>>(pc->partial + G, G, &pc->scal->rr);
      SPNET_CUDA_TRY(cudaMemcpyAsync(&h, pc->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s));
      SPNET_CUDA_TRY(cudaStreamSynchronize(s));
      const double tol = rtol * sqrt(h.bb);
      if (h.bb == 0.0) break;
      if (sqrt(h.rr) > tol && h.iter < maxit) {
        precond(pc, pc->r, pc->z, 1, nullptr, s);
        note_launch();
        k_direction<<<G, RED_BLOCK, 0, s>>>(N, pc->z, pc->p, pc->partial + 2 * G, pc->partial + 3 * G,
                                            G, pc->flexible, 1, pc->scal);
        for (;;) {
          for (int it = 0; it < chunk; ++it) iteration(pc, rtol, maxit, s);
          SPNET_CUDA_TRY(cudaMemcpyAsync(&h, pc->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s));
          SPNET_CUDA_TRY(cudaStreamSynchronize(s));
          if (h.done) break;
        }
      }
      // recompute the residual in FP64
      launch_spmv(pc->K, pc->x, pc->q, nullptr, G, pc->spmv_lanes, nullptr, s);
      note_launch();
      k_residual<<<G, RED_BLOCK, 0, s>>>(N, pc->b, pc->q, pc->vtmp, pc->partial + 4 * G);
      note_launch();
      k_reduce_to<<<1, 32, 0, s>>>(pc->partial + 4 * G, G, &pc->scal->rr_true);
      SPNET_CUDA_TRY(cudaMemcpyAsync(&h, pc->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s));
      SPNET_CUDA_TRY(cudaStreamSynchronize(s));
      const double rel = sqrt(h.rr_true) / sqrt(h.bb);
      if (rel <= rtol || restarts >= pc->max_restarts || h.iter >= maxit) break;
      ++restarts;
      int zero = 0;
      SPNET_CUDA_TRY(cudaMemcpyAsync(&pc->scal->done, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    }
    if (h.bb == 0.0) SPNET_CUDA_TRY(cudaMemsetAsync(pc->x, 0, sizeof(double) * N, s));
    note_launch();
    k_expand<<<G, 256, 0, s>>>(nd, op->free_of, pc->iperm, pc->x, gk, xk);
    cudaEventRecord(e1, s);
    SPNET_CUDA_TRY(cudaEventSynchronize(e1));
    const double rel = h.bb > 0.0 ? sqrt(h.rr_true) / sqrt(h.bb) : 0.0;
    const bool conv = h.bb == 0.0 || rel <= rtol;
    if (!conv) worst = SPNET_ERR_NO_CONVERGENCE;
    if (stats) {
      spnet_stats& st = stats[k];
      st = spnet_stats{};
      st.iterations = h.iter;
      st.restarts = restarts;
      st.converged = conv ? 1 : 0;
      st.status = conv ? SPNET_OK : SPNET_ERR_NO_CONVERGENCE;
      st.relres = rel;
      st.relres_recursive = h.bb > 0.0 ? sqrt(h.rr) / sqrt(h.bb) : 0.0;
      st.solve_ms = elapsed_ms(e0, e1);
    }
  }
  if (mem == SPNET_MEM_HOST)
    SPNET_TRY(copy_out(dx, x, sizeof(double) * nrhs * nd, mem, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SPNET_CUDA_TRY(cudaGetLastError());
  if (worst != SPNET_OK) return fail(worst, "pcg_solve: maxit reached before rtol");
  return SPNET_OK;
}

}  // namespace spnet
