// Preconditioned conjugate gradients (Section 4.2) on the free dofs in pc
// order, and the restriction / combination steps of B (Section 4.1).
//
// One iteration is five kernels; the star solves run on a second stream beside
// the coarse solve:
//   spmv_dir  p = z + beta p;  q = A z + beta q  (= A p);  (p, q) -> alpha
//   update    x += alpha p; r -= alpha q; |r|^2 -> stop test; per element the
//             Q1-weighted sums of r at its 2^d corners
//   coarse    z_c = A_0^{-1} R_0 r, R_0 r formed      | stars  w_j = A_j^{-1} E_j^T r
//             from the element sums in each block     |
//   combine   z = R_0^T z_c + sum_j E_j w_j; (r, z) [and (r, z_old)] -> beta
// Each reduction is finished by the last block of its kernel (fixed order:
// bitwise reproducible), which publishes the scalar for the next kernel.
// Every kernel returns at once when `done` is set, so chunks of iterations
// are captured once in a CUDA graph and replayed; the host reads the state
// only between chunks.
#include <cmath>

#include "spnet_internal.cuh"

namespace spnet {

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

// r = b - q and |r|^2 (or |b|^2 when q is null), finished by the last block
__global__ void k_residual(int64_t N, const double* b, const double* q, double* r, double* partial,
                           double* out, unsigned* cnt) {
  __shared__ double sh[32];
  double s = 0.0;
  GRID_STRIDE(i, N) {
    double v = q ? b[i] - q[i] : b[i];
    if (r) r[i] = v;
    s = fma(v, v, s);
  }
  block_partial(s, partial, sh);
  if (last_block(cnt)) {
    double t = block_sum(partial, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *out = t;
      *cnt = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// spmv_dir: p = z + beta p, q = A z + beta q, partials of (p, q); last block: alpha
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(256) k_spmv_dir(int64_t n, const int64_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ col,
                                                  const double* __restrict__ val,
                                                  const double* __restrict__ z, double* __restrict__ p,
                                                  double* __restrict__ q, double* partial, Scal* sc) {
  __shared__ double sh[32];
  pdl_wait();
  pdl_trigger();
  if (sc->done) return;
  const double beta = sc->beta;
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31;
  const int sub = lane % L;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t base = gwarp * RPW; base < n; base += nwarps * RPW) {
    const int64_t row = base + lane / L;
    const bool valid = row < n;
    // the row's own entries of z, p, q depend on nothing: load them first
    double zr = 0.0, pr = 0.0, qr = 0.0;
    if (valid && sub == 0) {
      zr = z[row];
      if (beta != 0.0) {
        pr = p[row];
        qr = q[row];
      }
    }
    double s = 0.0;
    if (valid) {
      const int64_t a = ptr[row], b = ptr[row + 1];
      for (int64_t k = a + sub; k < b; k += L) s = fma(val[k], __ldg(&z[col[k]]), s);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, L);
    if (valid && sub == 0) {
      const double pn = beta == 0.0 ? zr : fma(beta, pr, zr);
      const double qn = beta == 0.0 ? s : fma(beta, qr, s);
      p[row] = pn;
      q[row] = qn;
      dot = fma(pn, qn, dot);
    }
  }
  block_partial(dot, partial, sh);
  if (last_block(&sc->cnt[0])) {  // alpha = (r, z) / (p, q), for the update and the star solves
    const double pq = block_sum(partial, gridDim.x, sh);
    if (threadIdx.x == 0) {
      sc->pq = pq;
      sc->alpha = sc->rz / pq;
      sc->cnt[0] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// update (one warp per element): x += alpha p, rout = r - alpha q (mode 0; a
// different buffer, the star solves read r meanwhile) or r as is (mode 1);
// block partials of |r|^2; corner sums E[e][c][a] = sum_{p in e, comp a}
// phi_c(p) r_p.
// ---------------------------------------------------------------------------
template <int NC, int ND, class CT>
__global__ void __launch_bounds__(256, ND == 1 ? 4 : 2) k_update(int n_elem, int64_t N, const int32_t* __restrict__ elem_ptr,
                                                const int8_t* __restrict__ comp_of,
                                                const CT* __restrict__ xi, double* __restrict__ x,
                                                const double* __restrict__ r, double* __restrict__ rout,
                                                const double* __restrict__ p,
                                                const double* __restrict__ q, double* __restrict__ epart,
                                                double* partial, Scal* sc, int mode, int simplex) {
  constexpr int D = NC == 4 ? 2 : 3;
  __shared__ double sh[32];
  pdl_wait();
  pdl_trigger();
  if (mode == 0 && sc->done) return;
  const double alpha = mode == 0 ? sc->alpha : 0.0;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double rr = 0.0;
  for (int64_t e = gwarp; e < n_elem; e += nwarps) {
    CT acc[NC * ND];
#pragma unroll
    for (int t = 0; t < NC * ND; ++t) acc[t] = CT(0);
    const int a0 = elem_ptr[e], a1 = elem_ptr[e + 1];
    for (int i0 = a0; i0 < a1; i0 += 64) {
      // two dofs per lane; every load (from a valid address) before any use
      int ii[2];
      bool ok[2];
      double xv[2], pv[2], rv[2], qv[2];
      CT t[2][3];
      int cm[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        ii[h] = i0 + 32 * h + lane;
        ok[h] = ii[h] < a1;
        const int i = ok[h] ? ii[h] : a0;
        rv[h] = r[i];
        if (mode == 0) {
          xv[h] = x[i];
          pv[h] = p[i];
          qv[h] = q[i];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) t[h][a] = a < D ? __ldg(&xi[(int64_t)a * N + i]) : CT(0);
        cm[h] = ND == 1 ? 0 : comp_of[i];
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!ok[h]) continue;
        double v;
        if (mode == 0) {
          x[ii[h]] = fma(alpha, pv[h], xv[h]);
          v = fma(-alpha, qv[h], rv[h]);
          rout[ii[h]] = v;
        } else {
          v = rv[h];
        }
        rr = fma(v, v, rr);
        CT w[NC];
        basis_from_xi<NC>(t[h], w, simplex);
        const CT vc = (CT)v;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const CT wv = w[c] * vc;
          if (ND == 1) {
            acc[c] += wv;
          } else {  // selects, not an index: the accumulators stay in registers
#pragma unroll
            for (int b2 = 0; b2 < ND; ++b2) acc[c * ND + b2] += b2 == cm[h] ? wv : CT(0);
          }
        }
      }
    }
    constexpr int K = Pow2<NC * ND>::value;
    CT red[K];
#pragma unroll
    for (int t = 0; t < K; ++t) red[t] = t < NC * ND ? acc[t] : CT(0);
    const CT tot = reduce_scatter<K>(red, lane);
    const int ti = rs_index<K>(lane);
    if (rs_writer<K>(lane) && ti < NC * ND) epart[e * (NC * ND) + ti] = (double)tot;
  }
  block_partial(rr, partial, sh);  // |r|^2, summed by the last block of the combine
}

// r_c = R_0 r from the corner sums of the elements around each mesh node
__global__ void k_restrict(int n_mesh, Mesh m, int ndof, const double* __restrict__ epart,
                           const int32_t* __restrict__ cidx, double* __restrict__ rc, const int* done) {
  if (done && *done) return;
  GRID_STRIDE(ka, (int64_t)n_mesh * ndof) {
    const int ci = cidx[ka];
    if (ci < 0) continue;
    const int k = (int)(ka / ndof), a = (int)(ka % ndof);
    int km[3];
    mesh_multi(m, k, km);
    double s = 0.0;
    for (int cp = 0; cp < m.nc; ++cp) {
      const int e = elem_around(m, km, cp);
      if (e < 0) continue;
      const int c = (m.nc - 1) - cp;  // corner of e at mesh node k
      s += epart[((int64_t)e * m.nc + c) * ndof + a];
    }
    rc[ci] = s;
  }
}

// z = [R_0^T z_c] + [sum_j E_j w_j], one warp per element: the element's
// coarse values z_c at its corners and the bases of its entries in the star
// results are loaded once and held in registers; partials (r, z) and
// (r, z_old); last block: beta and, in a PCG step, |r|^2 from the update's
// partials, the iteration count and the stop test
template <int NC, int ND, class CT, class WS>
__global__ void __launch_bounds__(128, ND == 1 ? 7 : 4) k_combine(int n_elem, int64_t N, const int32_t* __restrict__ elem_ptr,
                                                 const int8_t* __restrict__ comp_of,
                                                 const CT* __restrict__ xi,
                                                 const int32_t* __restrict__ ecoarse,
                                                 const int64_t* __restrict__ estar,
                                                 const double* __restrict__ zc, const WS* __restrict__ w,
                                                 const double* __restrict__ r, double* __restrict__ z,
                                                 double* part1, double* part2, const double* __restrict__ prr,
                                                 int nrr, int with_coarse, int with_stars, Scal* sc,
                                                 int flexible, int first, int simplex) {
  constexpr int D = NC == 4 ? 2 : 3;
  __shared__ double sh[32];
  pdl_wait();
  pdl_trigger();
  if (sc && sc->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t e = gwarp; e < n_elem; e += nwarps) {
    CT zl = CT(0);
    int sl = -1;  // star bases fit 32 bits (checked at set-up)
    if (lane < NC * ND && with_coarse) {
      const int ci = ecoarse[e * (NC * ND) + lane];
      if (ci >= 0) zl = (CT)zc[ci];
    }
    if (lane < NC && with_stars) sl = (int)estar[e * NC + lane];
    // lane t keeps the coarse value of corner-component t; a dof fetches its
    // corners' values by shuffles (per-lane source: the dof's component)
    int sb[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) sb[c] = __shfl_sync(0xffffffffu, sl, c);
    const int a0 = elem_ptr[e], a1 = elem_ptr[e + 1];
    constexpr int U = 1;  // dofs per lane and pass (more would spill under the 64-register bound)
    for (int i0 = a0; i0 < a1; i0 += 32 * U) {
      // every load (from a valid address) before any use
      int ii[U];
      bool ok[U];
      CT t[U][3], wv[U][NC];
      double rv[U], zo[U];
      int cm[U];
#pragma unroll
      for (int h = 0; h < U; ++h) {
        ii[h] = i0 + 32 * h + lane;
        ok[h] = ii[h] < a1;
        const int i = ok[h] ? ii[h] : a0;
        const int off = i - a0;
        cm[h] = ND == 1 ? 0 : comp_of[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) t[h][a] = a < D ? __ldg(&xi[(int64_t)a * N + i]) : CT(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) wv[h][c] = (CT)__ldg(&w[sb[c] >= 0 ? sb[c] + off : 0]);
        rv[h] = sc ? __ldg(&r[i]) : 0.0;
        zo[h] = sc ? z[i] : 0.0;
      }
#pragma unroll
      for (int h = 0; h < U; ++h) {  // every lane computes (the shuffles need all lanes); valid ones write
        CT qw[NC];
        basis_from_xi<NC>(t[h], qw, simplex);
        CT vc = CT(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) vc = fma(qw[c], __shfl_sync(0xffffffffu, zl, c * ND + cm[h]), vc);
#pragma unroll
        for (int c = 0; c < NC; ++c) vc += sb[c] >= 0 ? wv[h][c] : CT(0);
        if (!ok[h]) continue;
        const double v = (double)vc;
        if (sc) {
          s1 = fma(rv[h], v, s1);
          s2 = fma(rv[h], zo[h], s2);
        }
        z[ii[h]] = v;
      }
    }
  }
  if (!sc) return;
  block_partial(s1, part1, sh);
  block_partial(s2, part2, sh);
  if (last_block(&sc->cnt[2])) {
    // in a PCG step also |r|^2 of the update, the iteration count and the stop test
    __shared__ double sh3[96];
    double tot[3];
    block_sum3(part1, gridDim.x, part2, gridDim.x, prr, first ? 0 : nrr, sh3, tot);
    const double rz_new = tot[0], rzo = tot[1], rr = tot[2];
    if (threadIdx.x == 0) {
      double beta = 0.0;
      if (!first) beta = flexible ? (rz_new - rzo) / sc->rz : rz_new / sc->rz;
      sc->beta = beta;
      sc->rz = rz_new;
      if (!first) {
        sc->rr = rr;
        sc->iter += 1;
        if (sqrt(rr) <= sc->rtol * sqrt(sc->bb) || sc->iter >= sc->maxit) sc->done = 1;
      }
      sc->cnt[2] = 0;
    }
  }
}

// per element and corner: the coarse index (per component) and the base of the
// element's entries in the star at that corner (-1 where there is none)
__global__ void k_elem_tables(int n_elem, Mesh m, int ndof, const int32_t* cidx, const int32_t* elem_star_off,
                              const int32_t* star_of_mesh, const int64_t* star_ptr, int32_t* ecoarse,
                              int64_t* estar) {
  GRID_STRIDE(e, (int64_t)n_elem) {
    for (int c = 0; c < m.nc; ++c) {
      const int k = mesh_of(m, (int)e, c);
      for (int a = 0; a < ndof; ++a) ecoarse[(e * m.nc + c) * ndof + a] = cidx[(int64_t)k * ndof + a];
      const int so = elem_star_off[e * m.nc + c];
      estar[e * m.nc + c] = so < 0 ? -1 : star_ptr[star_of_mesh[k]] + so;
    }
  }
}

int pc_elem_tables(spnet_pc_s* pc) {
  cudaStream_t s = pc->op->stream;
  SPNET_TRY(pc->mem.get(&pc->ecoarse, (size_t)pc->n_elem * pc->nc * pc->ndof));
  SPNET_TRY(pc->mem.get(&pc->estar, (size_t)pc->n_elem * pc->nc));
  note_launch();
  k_elem_tables<<<4 * num_sms(), 256, 0, s>>>(pc->n_elem, mesh_of_pc(pc), pc->ndof, pc->cidx, pc->elem_star_off,
                                              pc->star_of_mesh, pc->star_ptr, pc->ecoarse, pc->estar);
  SPNET_CUDA_TRY(cudaGetLastError());
  return SPNET_OK;
}

// one warp per element (blocks of `warps` warps), all resident at once when
// they fit; at most PG blocks (the stride of the partial-sum slots)
static int elem_grid(const spnet_pc_s* pc, int warps) {
  const int need = (pc->n_elem + warps - 1) / warps;
  return need < 1 ? 1 : need > pc->PG ? pc->PG : need;
}

template <int NC, int ND, class CT>
static void launch_update_t(spnet_pc_s* pc, const CT* xi, double* x, const double* r, double* rout,
                            const double* p, const double* q, Scal* sc, int mode, cudaStream_t s) {
  launch_pdl(k_update<NC, ND, CT>, elem_grid(pc, 8), 256, 0, s, pc->n_elem, pc->N, (const int32_t*)pc->elem_ptr,
             (const int8_t*)pc->comp_of, xi, x, r, rout, p, q, pc->epart, pc->partial + pc->PG, sc, mode,
             pc->coarse_space == SPNET_COARSE_P1 ? 1 : 0);
}

template <class CT>
static void launch_update_c(spnet_pc_s* pc, const CT* xi, double* x, const double* r, double* rout,
                            const double* p, const double* q, Scal* sc, int mode, cudaStream_t s) {
  if (pc->nc == 4 && pc->ndof == 1) launch_update_t<4, 1>(pc, xi, x, r, rout, p, q, sc, mode, s);
  else if (pc->nc == 8 && pc->ndof == 1) launch_update_t<8, 1>(pc, xi, x, r, rout, p, q, sc, mode, s);
  else if (pc->nc == 4) launch_update_t<4, 3>(pc, xi, x, r, rout, p, q, sc, mode, s);
  else launch_update_t<8, 3>(pc, xi, x, r, rout, p, q, sc, mode, s);
}

// mode 0: x += alpha p, rout = r - alpha q; mode 1: r as is (rout unused).
// exact: the corner sums in FP64 whatever the precision (the stand-alone
// restriction); otherwise in the arithmetic of the preconditioner
static void launch_update(spnet_pc_s* pc, double* x, const double* r, double* rout, const double* p,
                          const double* q, Scal* sc, int mode, cudaStream_t s, int exact = 0) {
  note_launch();
  ProfScope ps(KID_UPDATE, s);
  if (exact || pc->precision == SPNET_PREC_FP64) launch_update_c<double>(pc, pc->xi, x, r, rout, p, q, sc, mode, s);
  else launch_update_c<float>(pc, pc->xi32, x, r, rout, p, q, sc, mode, s);
}

// the SpMV's grid for its lanes per row: one row group per warp in a single pass, capped
// at 64 blocks per SM
int spmv_grid(const spnet_pc_s* pc, int lanes) {
  const int64_t want = (pc->N * lanes + 255) / 256;
  const int64_t cap = 64ll * num_sms();
  return (int)(want < 1 ? 1 : want > cap ? cap : want);
}

// Lanes per row of the SpMV, timed once per size class (half-octaves of the rows and of
// twice the mean row length, dofs per node) among half, once and twice the value the mean
// row length suggests; another value must beat that one by 5 %.  The choice changes the
// order of a row's sum, so every set-up of a class takes the one measured value.
int spmv_lanes_tune(spnet_pc_s* pc) {
  const int h = pc->spmv_lanes;
  if (pc->N < 65536) return SPNET_OK;  // a few microseconds whatever the choice
  const TuneClass key{{half_octave((double)pc->N), half_octave(2.0 * pc->K.nnz / pc->N), pc->ndof, 0}};
  int v = 0;
  if (tune_begin(TUNE_SPMV_LANES, key, &v)) {
    pc->spmv_lanes = v;
    pc->spmv_blocks = spmv_grid(pc, v);
    return SPNET_OK;
  }
  cudaStream_t s = pc->op->stream;
  int best = h, rc = SPNET_OK;
  float best_ms = 0.0f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMemsetAsync(pc->x, 0, sizeof(double) * pc->N, s) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    tune_end(TUNE_SPMV_LANES, key, 0);
    return fail(SPNET_ERR_CUDA, "setup_preconditioner: timing the SpMV failed");
  }
  for (int lanes : {h, h / 2, 2 * h}) {
    if (lanes < 1 || lanes > 32) continue;
    launch_spmv(pc->K, pc->x, pc->q, nullptr, pc->G, lanes, nullptr, s);  // warm-up
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 5; ++rep) launch_spmv(pc->K, pc->x, pc->q, nullptr, pc->G, lanes, nullptr, s);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = fail(SPNET_ERR_CUDA, "setup_preconditioner: timing the SpMV failed");
      break;
    }
    if (lanes == h || ms < 0.95f * best_ms) {
      best = lanes;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tune_end(TUNE_SPMV_LANES, key, rc == SPNET_OK ? best : 0);
  if (rc != SPNET_OK) return rc;
  pc->spmv_lanes = best;
  pc->spmv_blocks = spmv_grid(pc, best);
  return SPNET_OK;
}

static void launch_spmv_dir(spnet_pc_s* pc, cudaStream_t s) {
  note_launch();
  ProfScope ps(KID_SPMV, s);
  const Csr& A = pc->K;
  const int G = pc->spmv_blocks;
  double* part = pc->pspmv;
  auto go = [&](auto kernel) {
    launch_pdl(kernel, G, 256, 0, s, A.n, (const int64_t*)A.ptr, (const int32_t*)A.col, (const double*)A.val,
               (const double*)pc->z, pc->p, pc->q, part, pc->scal);
  };
  switch (pc->spmv_lanes) {
    case 1: go(k_spmv_dir<1>); break;
    case 2: go(k_spmv_dir<2>); break;
    case 4: go(k_spmv_dir<4>); break;
    case 8: go(k_spmv_dir<8>); break;
    case 16: go(k_spmv_dir<16>); break;
    default: go(k_spmv_dir<32>); break;
  }
}

void launch_restrict(spnet_pc_s* pc, double* rc, const int* done, cudaStream_t s) {
  if (pc->m0 == 0) return;
  note_launch();
  ProfScope ps(KID_RESTRICT, s);
  const int64_t n = (int64_t)pc->n_mesh * pc->ndof;
  int blocks = (int)((n + 255) / 256);
  if (blocks > pc->G) blocks = pc->G;
  k_restrict<<<blocks, 256, 0, s>>>(pc->n_mesh, mesh_of_pc(pc), pc->ndof, pc->epart, pc->cidx, rc, done);
}

template <int NC, int ND, class CT, class WS>
static void launch_combine_t(spnet_pc_s* pc, const CT* xi, const WS* w, const double* r, double* z,
                             int with_coarse, int with_stars, int dots, cudaStream_t s) {
  launch_pdl(k_combine<NC, ND, CT, WS>, elem_grid(pc, 4), 128, 0, s, pc->n_elem, pc->N,
             (const int32_t*)pc->elem_ptr, (const int8_t*)pc->comp_of, xi, (const int32_t*)pc->ecoarse,
             (const int64_t*)pc->estar, (const double*)pc->zc, w, r, z, pc->partial + 2 * pc->PG,
             pc->partial + 3 * pc->PG, (const double*)(pc->partial + pc->PG), elem_grid(pc, 8),
             (int)(with_coarse && pc->m0 > 0), (int)(with_stars && pc->S > 0), dots ? pc->scal : nullptr,
             pc->flexible, dots == 2 ? 1 : 0, pc->coarse_space == SPNET_COARSE_P1 ? 1 : 0);
}

template <class CT, class WS>
static void launch_combine_c(spnet_pc_s* pc, const CT* xi, const double* r, double* z, int with_coarse,
                             int with_stars, int dots, cudaStream_t s) {
  const WS* w = (const WS*)pc->w;
  if (pc->nc == 4 && pc->ndof == 1) launch_combine_t<4, 1>(pc, xi, w, r, z, with_coarse, with_stars, dots, s);
  else if (pc->nc == 8 && pc->ndof == 1) launch_combine_t<8, 1>(pc, xi, w, r, z, with_coarse, with_stars, dots, s);
  else if (pc->nc == 4) launch_combine_t<4, 3>(pc, xi, w, r, z, with_coarse, with_stars, dots, s);
  else launch_combine_t<8, 3>(pc, xi, w, r, z, with_coarse, with_stars, dots, s);
}

// dots: 0 none, 1 PCG step (beta from the previous rz), 2 PCG start (beta = 0).
// exact: the prolongation in FP64 whatever the precision (the stand-alone
// prolongation); otherwise in the arithmetic of the preconditioner
void launch_combine(spnet_pc_s* pc, const double* r, double* z, int with_coarse, int with_stars, int dots,
                    cudaStream_t s, int exact) {
  note_launch();
  ProfScope ps(KID_COMBINE, s);
  if (pc->precision == SPNET_PREC_FP64)
    launch_combine_c<double, double>(pc, pc->xi, r, z, with_coarse, with_stars, dots, s);
  else if (exact)
    launch_combine_c<double, float>(pc, pc->xi, r, z, with_coarse, with_stars, dots, s);
  else
    launch_combine_c<float, float>(pc, pc->xi32, r, z, with_coarse, with_stars, dots, s);
}

// z = B r for a vector r already in pc order (corner sums of r computed here)
static void precond_any(spnet_pc_s* pc, double* r, double* z, int with_coarse, int with_stars, int dots,
                        cudaStream_t s) {
  if (with_coarse && pc->m0 > 0) {
    launch_update(pc, nullptr, r, nullptr, nullptr, nullptr, pc->scal, 1, s);
    launch_coarse_apply(pc, nullptr, pc->zc, nullptr, s);  // restriction fused
  }
  if (with_stars) launch_star_solve(pc, r, nullptr, nullptr, nullptr, s);
  launch_combine(pc, r, z, with_coarse, with_stars, dots, s);
}

// one PCG iteration; the star solves go to the side stream when `side` is set.
// The residual alternates between pc->r and pc->r2 (parity): the update writes
// the new residual into the other buffer while the star solves, started right
// after the SpMV, form the same values from the old residual, q and alpha.
// spnet_pc_record_iterates: x^(l) in free order at buf + l N, l = the step count
__global__ void k_record_iterate(int64_t N, const int32_t* perm, const double* xp, const Scal* sc, double* buf,
                                 int64_t max) {
  const int64_t l = sc->iter;
  if (l >= max) return;
  double* out = buf + l * N;
  GRID_STRIDE(p, N) out[perm[p]] = xp[p];
}

static void record_iterate(spnet_pc_s* pc, cudaStream_t s) {
  if (!pc->rec_buf) return;
  note_launch();
  k_record_iterate<<<pc->G, 256, 0, s>>>(pc->N, pc->perm, pc->x, pc->scal, pc->rec_buf, pc->rec_max);
}

static void iteration(spnet_pc_s* pc, cudaStream_t s, cudaStream_t side, int parity) {
  const int* done = &pc->scal->done;
  double* rc = parity ? pc->r2 : pc->r;  // residual of the previous iteration
  double* rn = parity ? pc->r : pc->r2;  // residual of this one
  launch_spmv_dir(pc, s);
  if (side) {
    cudaEventRecord(pc->ev_fork, s);
    cudaStreamWaitEvent(side, pc->ev_fork, 0);
    launch_star_solve(pc, rc, pc->q, pc->scal, done, side);
    cudaEventRecord(pc->ev_join, side);
  } else {
    launch_star_solve(pc, rc, pc->q, pc->scal, done, s);
  }
  launch_update(pc, pc->x, rc, rn, pc->p, pc->q, pc->scal, 0, s);
  launch_coarse_apply(pc, nullptr, pc->zc, done, s);  // restriction fused
  if (side) cudaStreamWaitEvent(s, pc->ev_join, 0);
  launch_combine(pc, rn, pc->z, 1, 1, 1, s);
}

constexpr int CHUNK = 8;  // even: a chunk leaves the residual in pc->r
static_assert(CHUNK % 2 == 0, "the residual buffers alternate per iteration");

// the chunk of iterations as a CUDA graph (captured once per preconditioner)
static int chunk_graph(spnet_pc_s* pc, cudaStream_t s) {
  if (pc->graph_exec) return SPNET_OK;
  if (!pc->side) {
    SPNET_CUDA_TRY(cudaStreamCreateWithFlags(&pc->side, cudaStreamNonBlocking));
    SPNET_CUDA_TRY(cudaEventCreateWithFlags(&pc->ev_fork, cudaEventDisableTiming));
    SPNET_CUDA_TRY(cudaEventCreateWithFlags(&pc->ev_join, cudaEventDisableTiming));
  }
  cudaGraph_t g = nullptr;
  SPNET_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const long long before = launch_count();
  for (int it = 0; it < CHUNK; ++it) iteration(pc, s, pc->side, it & 1);
  pc->graph_launches = (int)(launch_count() - before);
  add_launches(-pc->graph_launches);  // captured, not launched
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return fail(SPNET_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&pc->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    pc->graph_exec = nullptr;
    return fail(SPNET_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  return SPNET_OK;
}

static int run_chunk(spnet_pc_s* pc, cudaStream_t s) {
  if (profiling_on() || pc->rec_buf) {
    // eager launches so that every kernel can be timed with its own events, and
    // the iterate of every step can be recorded
    for (int it = 0; it < CHUNK; ++it) {
      iteration(pc, s, nullptr, it & 1);
      record_iterate(pc, s);
    }
    return SPNET_OK;
  }
  SPNET_TRY(chunk_graph(pc, s));
  add_launches(pc->graph_launches);
  SPNET_CUDA_TRY(cudaGraphLaunch(pc->graph_exec, s));
  return SPNET_OK;
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
    case SPNET_EXPORT_STAR_CORE:
      if (pc->S) SPNET_CUDA_TRY(cudaMemcpyAsync(host_buf, pc->star_core, sizeof(int32_t) * pc->S, cudaMemcpyDeviceToHost, s));
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
  to_pc(pc, r_free, pc->vtmp);
  if (which == 0) precond_any(pc, pc->vtmp, pc->z, 1, 1, 0, s);
  else if (which == 1) precond_any(pc, pc->vtmp, pc->z, 1, 0, 0, s);
  else precond_any(pc, pc->vtmp, pc->z, 0, 1, 0, s);
  from_pc(pc, pc->z, z_free);
  SPNET_CUDA_TRY(cudaGetLastError());
  return SPNET_OK;
}

int pc_restrict_free(spnet_pc_s* pc, const double* r_free, double* rc) {
  cudaStream_t s = pc->op->stream;
  to_pc(pc, r_free, pc->vtmp);
  if (pc->m0 == 0) return SPNET_OK;
  launch_update(pc, nullptr, pc->vtmp, nullptr, nullptr, nullptr, pc->scal, 1, s, 1);
  launch_restrict(pc, rc, nullptr, s);
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
  const int kmax = star_batch_max_k(pc);
  const int kb = pc->batch_rhs < kmax ? pc->batch_rhs : kmax;
  if (nrhs >= 2 && kb >= 2) {  // blocks of right-hand sides stepped together
    int worst = SPNET_OK;
    for (int k0 = 0; k0 < nrhs; k0 += kb) {
      const int kk = nrhs - k0 < kb ? nrhs - k0 : kb;
      const double* fk = df + (int64_t)k0 * nd;
      const double* gk = dg + (int64_t)k0 * ndir;
      double* xk = dx + (int64_t)k0 * nd;
      spnet_stats* sk = stats ? stats + k0 : nullptr;
      const int rc = kk >= 2 ? pcg_batch_run(op, pc, kk, fk, gk, xk, use_x0, rtol, maxit, sk)
                             : pcg_run(op, pc, 1, fk, gk, xk, use_x0, rtol, maxit, SPNET_MEM_DEVICE, sk);
      if (rc == SPNET_ERR_NO_CONVERGENCE) worst = rc;
      else if (rc != SPNET_OK) return rc;
    }
    if (mem == SPNET_MEM_HOST) SPNET_TRY(copy_out(dx, x, sizeof(double) * nrhs * nd, mem, s));
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));
    if (worst != SPNET_OK) return fail(worst, "pcg_solve: maxit reached before rtol");
    return SPNET_OK;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int worst = SPNET_OK;
  unsigned* cnt3 = &pc->scal->cnt[3];
  for (int k = 0; k < nrhs; ++k) {
    const double* fk = df + (int64_t)k * nd;
    const double* gk = dg + (int64_t)k * ndir;
    double* xk = dx + (int64_t)k * nd;
    cudaEventRecord(e0, s);
    Scal init{};
    init.rtol = rtol;
    init.maxit = maxit;
    SPNET_CUDA_TRY(cudaMemcpyAsync(pc->scal, &init, sizeof(Scal), cudaMemcpyHostToDevice, s));
    note_launch();
    k_build_rhs<<<G, 256, 0, s>>>(N, pc->perm, op->free_dofs, fk, op->fd.ptr, op->fd.col, op->fd.val,
                                  gk, pc->b);
    note_launch();
    k_residual<<<G, 256, 0, s>>>(N, pc->b, nullptr, nullptr, pc->partial, &pc->scal->bb, cnt3);
    if (use_x0) {
      note_launch();
      k_x0_from_dofs<<<G, 256, 0, s>>>(N, pc->perm, op->free_dofs, xk, pc->x);
      launch_spmv(pc->K, pc->x, pc->q, nullptr, G, pc->spmv_lanes, nullptr, s);
    } else {
      SPNET_CUDA_TRY(cudaMemsetAsync(pc->x, 0, sizeof(double) * N, s));
      SPNET_CUDA_TRY(cudaMemsetAsync(pc->q, 0, sizeof(double) * N, s));
    }
    record_iterate(pc, s);  // l = 0
    int restarts = 0;
    Scal h{};
    for (;;) {
      // (re)start: r = b - A x, z = B r, beta = 0
      note_launch();
      k_residual<<<G, 256, 0, s>>>(N, pc->b, pc->q, pc->r, pc->partial, &pc->scal->rr, cnt3);
      SPNET_CUDA_TRY(cudaMemcpyAsync(&h, pc->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s));
      SPNET_CUDA_TRY(cudaStreamSynchronize(s));
      if (!std::isfinite(h.bb) || !std::isfinite(h.rr)) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(SPNET_ERR_BAD_INPUT, std::isfinite(h.bb)
                                             ? "pcg_solve: non-finite initial guess"
                                             : "pcg_solve: non-finite right-hand side or Dirichlet data");
      }
      const double tol = rtol * sqrt(h.bb);
      if (h.bb == 0.0) break;
      if (sqrt(h.rr) > tol && h.iter < maxit) {
        precond_any(pc, pc->r, pc->z, 1, 1, 2, s);  // z = B r, rz = (r, z), beta = 0
        for (;;) {
          SPNET_TRY(run_chunk(pc, s));
          SPNET_CUDA_TRY(cudaMemcpyAsync(&h, pc->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s));
          SPNET_CUDA_TRY(cudaStreamSynchronize(s));
          if (h.done) break;
        }
      }
      // recompute the residual in FP64
      launch_spmv(pc->K, pc->x, pc->q, nullptr, G, pc->spmv_lanes, nullptr, s);
      note_launch();
      k_residual<<<G, 256, 0, s>>>(N, pc->b, pc->q, pc->vtmp, pc->partial, &pc->scal->rr_true, cnt3);
      SPNET_CUDA_TRY(cudaMemcpyAsync(&h, pc->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s));
      SPNET_CUDA_TRY(cudaStreamSynchronize(s));
      const double rel = sqrt(h.rr_true) / sqrt(h.bb);
      if (rel <= rtol || restarts >= pc->max_restarts || h.iter >= maxit) break;
      ++restarts;
      int zero = 0;
      SPNET_CUDA_TRY(cudaMemcpyAsync(&pc->scal->done, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
      SPNET_CUDA_TRY(cudaStreamSynchronize(s));
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
