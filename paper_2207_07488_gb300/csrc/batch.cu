// PCG for k right-hand sides at once (2 <= k <= 32) on one operator and one
// preconditioner (Section 4.2, the same iteration per right-hand side).
//
// The k systems step together; their vectors are blocks [dof][k] (right-hand
// side fastest), so the SpMV reads each entry of A once for all k, the
// preconditioner reads its factors and coarse tiles once for all k, and every
// kernel keeps k independent sums.  A right-hand side that has met its
// tolerance is frozen (alpha = 0) while the others finish.  Each right-hand
// side keeps its own scalars and every sum is taken in an order fixed by the
// padded block width kp (k rounded up to a power of two), so a right-hand
// side gives the same bits in any block of the same width.
//
// One iteration is five kernels, the star solves on a second stream beside
// the coarse solve:
//   spmm_dir  P = Z + beta P; Q = A Z + beta Q; (p_j, q_j) -> alpha_j
//   update    X += alpha P; R -= alpha Q; |r_j|^2; Q1-weighted corner sums per column
//   coarse    Z_c = A_0^{-1} R_0 R, each tile once for all columns | stars, lane j = column j
//   combine   Z = R_0^T Z_c + sum_j E_j W_j; (r_j, z_j), (r_j, z_old_j) -> beta_j, stop tests
#include <cmath>
#include <vector>

#include "spnet_internal.cuh"

namespace spnet {

constexpr int KMAX = 32;

// per right-hand side scalars of the batch (one writer per kernel: its last block)
struct BScal {
  double rz[KMAX], pq[KMAX], rr[KMAX], bb[KMAX], alpha[KMAX], beta[KMAX];
  int done[KMAX], iters[KMAX];
  double rtol;
  int k, maxit, iter, all_done;
  unsigned cnt[4];
};

static inline int pow2_at_least(int k) {
  return k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
}

// sum over the lanes that share a column (lanes j, j + kp, j + 2 kp, ...); fixed order
__device__ __forceinline__ double column_lanes_sum(double v, int kp) {
  for (int o = kp; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block partials of one value per column: part[block][KMAX]
__device__ __forceinline__ void column_partials(double v, int kp, double* part, double (*sh)[KMAX]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = column_lanes_sum(v, kp);
  if (lane < kp) sh[wid][lane] = v;
  __syncthreads();
  if ((int)threadIdx.x < kp) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w][threadIdx.x];
    part[(int64_t)blockIdx.x * KMAX + threadIdx.x] = t;
  }
  __syncthreads();
}

// sum over nb blocks of column j's partials (by one warp; every lane gets it); fixed order
__device__ __forceinline__ double column_total(const double* part, int nb, int j) {
  double t = 0.0;
  for (int b = threadIdx.x & 31; b < nb; b += 32) t += __ldcg(&part[(int64_t)b * KMAX + j]);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// P = Z + beta P, Q = A Z + beta Q per column; partials of (p_j, q_j); last block: alpha_j
__global__ void __launch_bounds__(256) k_bspmm_dir(int64_t n, int k, int kp, const int64_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ col, const double* __restrict__ val,
                                                   const double* __restrict__ Z, double* __restrict__ P,
                                                   double* __restrict__ Q, double* part, BScal* bs) {
  __shared__ double sh[8][KMAX];
  pdl_wait();
  pdl_trigger();
  if (bs->all_done) return;
  const int lane = threadIdx.x & 31;
  const int rows = 32 / kp, r = lane / kp, j = lane % kp;
  const bool act = j < k;
  const double beta = act ? bs->beta[j] : 0.0;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  if (act) {
    for (int64_t row = gw * rows + r; row < n; row += nw * rows) {
      double s = 0.0;
      for (int64_t q = ptr[row]; q < ptr[row + 1]; ++q) s = fma(val[q], Z[(int64_t)col[q] * k + j], s);
      const int64_t o = row * k + j;
      const double z = Z[o];
      const double pn = beta == 0.0 ? z : fma(beta, P[o], z);
      const double qn = beta == 0.0 ? s : fma(beta, Q[o], s);
      P[o] = pn;
      Q[o] = qn;
      dot = fma(pn, qn, dot);
    }
  }
  column_partials(dot, kp, part, sh);
  if (last_block(&bs->cnt[0])) {
    for (int jj = threadIdx.x >> 5; jj < k; jj += (int)(blockDim.x >> 5)) {
      const double pq = column_total(part, gridDim.x, jj);
      if ((threadIdx.x & 31) == 0) {
        bs->pq[jj] = pq;
        bs->alpha[jj] = (bs->done[jj] || pq == 0.0) ? 0.0 : bs->rz[jj] / pq;
      }
    }
    if (threadIdx.x == 0) bs->cnt[0] = 0;
  }
}

// one warp per element, lanes (row r, column j); mode 0: X += alpha P, R -= alpha Q;
// mode 1: R as is.  Partials of |r_j|^2; corner sums EP[(e, corner, comp)][j] of
// phi_c r_j.  A lane takes BU of the element's dofs at a time, every load first.
constexpr int BU = 4;

template <int NC, int ND, class CT>
__global__ void __launch_bounds__(256) k_bupdate(int n_elem, int64_t N, int k, int kp,
                                                 const int32_t* __restrict__ elem_ptr,
                                                 const int8_t* __restrict__ comp_of, const CT* __restrict__ xi,
                                                 double* __restrict__ X, double* __restrict__ R,
                                                 const double* __restrict__ P, const double* __restrict__ Q,
                                                 double* __restrict__ EP, double* part, BScal* bs, int mode,
                                                 int simplex) {
  constexpr int D = NC == 4 ? 2 : 3;
  __shared__ double sh[8][KMAX];
  pdl_wait();
  pdl_trigger();
  if (mode == 0 && bs->all_done) return;
  const int lane = threadIdx.x & 31;
  const int rows = 32 / kp, r = lane / kp, j = lane % kp;
  const bool act = j < k;
  const double alpha = (mode == 0 && act) ? bs->alpha[j] : 0.0;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double rr = 0.0;
  for (int64_t e = gw; e < n_elem; e += nw) {
    CT acc[NC * ND];
#pragma unroll
    for (int t = 0; t < NC * ND; ++t) acc[t] = CT(0);
    const int a0 = elem_ptr[e], a1 = elem_ptr[e + 1];
    if (act) {
      for (int i0 = a0 + r; i0 < a1; i0 += rows * BU) {
        bool ok[BU];
        int ii[BU], cm[BU];
        double xv[BU], pv[BU], qv[BU], rv[BU];
        CT t[BU][3];
#pragma unroll
        for (int u = 0; u < BU; ++u) {
          ii[u] = i0 + u * rows;
          ok[u] = ii[u] < a1;
          const int i = ok[u] ? ii[u] : a0;
          const int64_t o = (int64_t)i * k + j;
          rv[u] = R[o];
          if (mode == 0) {
            xv[u] = X[o];
            pv[u] = P[o];
            qv[u] = Q[o];
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) t[u][a] = a < D ? __ldg(&xi[(int64_t)a * N + i]) : CT(0);
          cm[u] = ND == 1 ? 0 : comp_of[i];
        }
#pragma unroll
        for (int u = 0; u < BU; ++u) {
          if (!ok[u]) continue;
          const int64_t o = (int64_t)ii[u] * k + j;
          double v = rv[u];
          if (mode == 0) {
            X[o] = fma(alpha, pv[u], xv[u]);
            v = fma(-alpha, qv[u], v);
            R[o] = v;
          }
          rr = fma(v, v, rr);
          CT w[NC];
          basis_from_xi<NC>(t[u], w, simplex);
          const CT vc = (CT)v;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const CT wv = w[c] * vc;
#pragma unroll
            for (int b2 = 0; b2 < ND; ++b2) acc[c * ND + b2] += b2 == cm[u] ? wv : CT(0);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < NC * ND; ++t) {
      CT v = acc[t];
      for (int o = kp; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (r == 0 && act) EP[(e * (NC * ND) + t) * k + j] = (double)v;
    }
  }
  column_partials(rr, kp, part, sh);
}

// one warp per element: Z = R_0^T Z_c + sum_j E_j W_j per column; with dots,
// partials of (r_j, z_j), (r_j, z_old_j) and in the last block beta_j, |r_j|^2
// (from the update's partials), the stop tests (dots 1: a PCG step; 2: the start)
template <int NC, int ND, class CT, class WS>
__global__ void __launch_bounds__(256) k_bcombine(int n_elem, int64_t N, int k, int kp,
                                                  const int32_t* __restrict__ elem_ptr,
                                                  const int8_t* __restrict__ comp_of, const CT* __restrict__ xi,
                                                  const int32_t* __restrict__ ecoarse,
                                                  const int64_t* __restrict__ estar, const double* __restrict__ ZC,
                                                  const WS* __restrict__ W, const double* __restrict__ R,
                                                  double* __restrict__ Z, double* part1, double* part2,
                                                  const double* prr, int nrr, int with_coarse, int with_stars,
                                                  BScal* bs, int dots, int flexible, int simplex) {
  constexpr int D = NC == 4 ? 2 : 3;
  __shared__ double sh[8][KMAX];
  pdl_wait();
  pdl_trigger();
  if (dots == 1 && bs->all_done) return;
  const int lane = threadIdx.x & 31;
  const int rows = 32 / kp, r = lane / kp, j = lane % kp;
  const bool act = j < k;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t e = gw; e < n_elem; e += nw) {
    if (!act) continue;
    CT zcv[NC * ND];
#pragma unroll
    for (int t = 0; t < NC * ND; ++t) {
      CT v = CT(0);
      if (with_coarse) {
        const int ci = ecoarse[e * (NC * ND) + t];
        if (ci >= 0) v = (CT)ZC[(int64_t)ci * k + j];
      }
      zcv[t] = v;
    }
    int sb[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) sb[c] = with_stars ? (int)estar[e * NC + c] : -1;
    const int a0 = elem_ptr[e], a1 = elem_ptr[e + 1];
    for (int i0 = a0 + r; i0 < a1; i0 += rows * BU) {
      bool ok[BU];
      int ii[BU], cm[BU];
      CT t[BU][3], wv[BU][NC];
      double rv[BU], zo[BU];
#pragma unroll
      for (int u = 0; u < BU; ++u) {
        ii[u] = i0 + u * rows;
        ok[u] = ii[u] < a1;
        const int i = ok[u] ? ii[u] : a0;
        const int off = i - a0;
#pragma unroll
        for (int a = 0; a < 3; ++a) t[u][a] = a < D ? __ldg(&xi[(int64_t)a * N + i]) : CT(0);
        cm[u] = ND == 1 ? 0 : comp_of[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) wv[u][c] = sb[c] >= 0 ? (CT)__ldg(&W[(int64_t)(sb[c] + off) * k + j]) : CT(0);
        const int64_t o = (int64_t)i * k + j;
        rv[u] = dots ? __ldg(&R[o]) : 0.0;
        zo[u] = dots ? Z[o] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < BU; ++u) {
        if (!ok[u]) continue;
        CT w[NC];
        basis_from_xi<NC>(t[u], w, simplex);
        CT v = CT(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          CT zv = zcv[c * ND];
#pragma unroll
          for (int b2 = 1; b2 < ND; ++b2) zv = b2 == cm[u] ? zcv[c * ND + b2] : zv;
          v = fma(w[c], zv, v);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) v += wv[u][c];
        const double vd = (double)v;
        if (dots) {
          s1 = fma(rv[u], vd, s1);
          s2 = fma(rv[u], zo[u], s2);
        }
        Z[(int64_t)ii[u] * k + j] = vd;
      }
    }
  }
  if (!dots) return;
  column_partials(s1, kp, part1, sh);
  column_partials(s2, kp, part2, sh);
  if (last_block(&bs->cnt[2])) {
    for (int jj = threadIdx.x >> 5; jj < k; jj += (int)(blockDim.x >> 5)) {
      const double rz_new = column_total(part1, gridDim.x, jj);
      const double rzo = column_total(part2, gridDim.x, jj);
      const double rr = dots == 1 ? column_total(prr, nrr, jj) : 0.0;
      if ((threadIdx.x & 31) == 0) {
        if (dots == 2) {  // PCG start: beta = 0
          bs->beta[jj] = 0.0;
          bs->rz[jj] = rz_new;
        } else if (!bs->done[jj]) {
          const double rz = bs->rz[jj];
          bs->beta[jj] = rz == 0.0 ? 0.0 : (flexible ? (rz_new - rzo) / rz : rz_new / rz);
          bs->rz[jj] = rz_new;
          bs->rr[jj] = rr;
          bs->iters[jj] = bs->iter + 1;
          if (sqrt(rr) <= bs->rtol * sqrt(bs->bb[jj]) || bs->iter + 1 >= bs->maxit) bs->done[jj] = 1;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (dots == 1) bs->iter += 1;
      int all = 1;
      for (int jj = 0; jj < k; ++jj) all &= bs->done[jj];
      bs->all_done = all;
      bs->cnt[2] = 0;
    }
  }
}

// column j of a block [N][k] <-> a vector of length N (pc order)
__global__ void k_col_put(int64_t N, int k, int j, const double* __restrict__ v, double* __restrict__ B) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    B[i * k + j] = v[i];
}
__global__ void k_col_get(int64_t N, int k, int j, const double* __restrict__ B, double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = B[i * k + j];
}

// [k][N] in free order (one right-hand side after another) <-> [N][k] in pc order
__global__ void k_cols_to_pc(int64_t N, int k, const int32_t* __restrict__ perm, const double* __restrict__ v,
                             double* __restrict__ B) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N * k; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = q / k;
    const int j = (int)(q % k);
    B[q] = v[(int64_t)j * N + perm[p]];
  }
}
__global__ void k_cols_from_pc(int64_t N, int k, const int32_t* __restrict__ perm, const double* __restrict__ B,
                               double* __restrict__ v) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N * k; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = q / k;
    const int j = (int)(q % k);
    v[(int64_t)j * N + perm[p]] = B[q];
  }
}

// the device state of a batch
struct Batch {
  int k = 0, kp = 0;
  double *X = nullptr, *R = nullptr, *P = nullptr, *Q = nullptr, *Z = nullptr, *EP = nullptr, *ZC = nullptr;
  void *W = nullptr, *cpart = nullptr;
  double *p0 = nullptr, *p1 = nullptr, *p2 = nullptr, *p3 = nullptr;  // partials [blocks][KMAX]
  BScal* bs = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// the block vectors of k right-hand sides (iterate: also X, P, Q)
static int batch_alloc(spnet_pc_s* pc, Batch& b, int k, DevArena& tmp, bool iterate) {
  const int64_t N = pc->N;
  b.k = k;
  b.kp = pow2_at_least(k);
  const int vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  const int64_t nep = (int64_t)pc->n_elem * pc->nc * pc->ndof;
  const int64_t nk = (N > 0 ? N : 1) * k;
  if (iterate) {
    SPNET_TRY(tmp.get(&b.X, nk));
    SPNET_TRY(tmp.get(&b.P, nk));
    SPNET_TRY(tmp.get(&b.Q, nk));
  }
  SPNET_TRY(tmp.get(&b.R, nk));
  SPNET_TRY(tmp.get(&b.Z, nk));
  SPNET_TRY(tmp.get(&b.EP, (nep > 0 ? nep : 1) * k));
  SPNET_TRY(tmp.get(&b.ZC, (int64_t)(pc->m0 > 0 ? pc->m0 : 1) * k));
  SPNET_TRY(tmp.alloc(&b.W, (size_t)(pc->sum_s > 0 ? pc->sum_s : 1) * k * vb));
  SPNET_TRY(tmp.alloc(&b.cpart, pc->m0 > 0 ? coarse_batch_part_bytes(pc, k) : 16));
  SPNET_TRY(tmp.get(&b.p0, (int64_t)pc->PG * KMAX));
  SPNET_TRY(tmp.get(&b.p1, (int64_t)pc->PG * KMAX));
  SPNET_TRY(tmp.get(&b.p2, (int64_t)pc->PG * KMAX));
  SPNET_TRY(tmp.get(&b.p3, (int64_t)pc->PG * KMAX));
  SPNET_TRY(tmp.get(&b.bs, 1));
  SPNET_CUDA_TRY(cudaMemsetAsync(b.bs, 0, sizeof(BScal), tmp.stream));
  return SPNET_OK;
}

// blocks of 8 warps, one element per warp, at most PG (the stride of the partial slots)
static int elem_blocks(const spnet_pc_s* pc) {
  const int need = (pc->n_elem + 7) / 8;
  return need < 1 ? 1 : need > pc->PG ? pc->PG : need;
}

template <int NC, int ND, class CT>
static void bupdate_t(spnet_pc_s* pc, Batch& b, const CT* xi, int mode, cudaStream_t s) {
  launch_pdl(k_bupdate<NC, ND, CT>, elem_blocks(pc), 256, 0, s, pc->n_elem, pc->N, b.k, b.kp,
             (const int32_t*)pc->elem_ptr, (const int8_t*)pc->comp_of, xi, b.X, b.R, (const double*)b.P,
             (const double*)b.Q, b.EP, b.p1, b.bs, mode, pc->coarse_space == SPNET_COARSE_P1 ? 1 : 0);
}

template <class CT>
static void bupdate_c(spnet_pc_s* pc, Batch& b, const CT* xi, int mode, cudaStream_t s) {
  if (pc->nc == 4 && pc->ndof == 1) bupdate_t<4, 1>(pc, b, xi, mode, s);
  else if (pc->nc == 8 && pc->ndof == 1) bupdate_t<8, 1>(pc, b, xi, mode, s);
  else if (pc->nc == 4) bupdate_t<4, 3>(pc, b, xi, mode, s);
  else bupdate_t<8, 3>(pc, b, xi, mode, s);
}

static void launch_bupdate(spnet_pc_s* pc, Batch& b, int mode, cudaStream_t s) {
  note_launch();
  ProfScope ps(KID_UPDATE, s);
  if (pc->precision == SPNET_PREC_FP64) bupdate_c<double>(pc, b, pc->xi, mode, s);
  else bupdate_c<float>(pc, b, pc->xi32, mode, s);
}

template <int NC, int ND, class CT, class WS>
static void bcombine_t(spnet_pc_s* pc, Batch& b, const CT* xi, int wc, int ws, int dots, cudaStream_t s) {
  launch_pdl(k_bcombine<NC, ND, CT, WS>, elem_blocks(pc), 256, 0, s, pc->n_elem, pc->N, b.k, b.kp,
             (const int32_t*)pc->elem_ptr, (const int8_t*)pc->comp_of, xi, (const int32_t*)pc->ecoarse,
             (const int64_t*)pc->estar, (const double*)b.ZC, (const WS*)b.W, (const double*)b.R, b.Z, b.p2, b.p3,
             (const double*)b.p1, elem_blocks(pc), (int)(wc && pc->m0 > 0), (int)(ws && pc->S > 0), b.bs, dots,
             pc->flexible, pc->coarse_space == SPNET_COARSE_P1 ? 1 : 0);
}

template <class CT, class WS>
static void bcombine_c(spnet_pc_s* pc, Batch& b, const CT* xi, int wc, int ws, int dots, cudaStream_t s) {
  if (pc->nc == 4 && pc->ndof == 1) bcombine_t<4, 1, CT, WS>(pc, b, xi, wc, ws, dots, s);
  else if (pc->nc == 8 && pc->ndof == 1) bcombine_t<8, 1, CT, WS>(pc, b, xi, wc, ws, dots, s);
  else if (pc->nc == 4) bcombine_t<4, 3, CT, WS>(pc, b, xi, wc, ws, dots, s);
  else bcombine_t<8, 3, CT, WS>(pc, b, xi, wc, ws, dots, s);
}

static void launch_bcombine(spnet_pc_s* pc, Batch& b, int dots, cudaStream_t s, int wc = 1, int ws = 1) {
  note_launch();
  ProfScope ps(KID_COMBINE, s);
  if (pc->precision == SPNET_PREC_FP64) bcombine_c<double, double>(pc, b, pc->xi, wc, ws, dots, s);
  else bcombine_c<float, float>(pc, b, pc->xi32, wc, ws, dots, s);
}

static void launch_bspmm(spnet_pc_s* pc, Batch& b, cudaStream_t s) {
  note_launch();
  ProfScope ps(KID_SPMV, s);
  const int64_t want = (pc->N * b.kp + 255) / 256;
  const int grid = (int)(want < 1 ? 1 : want > pc->PG ? pc->PG : want);
  launch_pdl(k_bspmm_dir, grid, 256, 0, s, pc->K.n, b.k, b.kp, (const int64_t*)pc->K.ptr,
             (const int32_t*)pc->K.col, (const double*)pc->K.val, (const double*)b.Z, b.P, b.Q, b.p0, b.bs);
}

// Z = B R for the whole block and the start scalars (beta = 0, rz_j = (r_j, z_j))
static int precond_batch(spnet_pc_s* pc, Batch& b, cudaStream_t s) {
  launch_bupdate(pc, b, 1, s);
  SPNET_TRY(launch_coarse_batch(pc, b.EP, b.k, b.ZC, b.cpart, nullptr, s));
  SPNET_TRY(launch_star_batch(pc, b.R, b.k, b.W, nullptr, s));
  launch_bcombine(pc, b, 2, s);
  return SPNET_OK;
}

static int batch_iteration(spnet_pc_s* pc, Batch& b, cudaStream_t s, cudaStream_t side) {
  const int* done = &b.bs->all_done;
  launch_bspmm(pc, b, s);
  launch_bupdate(pc, b, 0, s);
  if (side) {
    SPNET_CUDA_TRY(cudaEventRecord(b.ev_fork, s));
    SPNET_CUDA_TRY(cudaStreamWaitEvent(side, b.ev_fork, 0));
    SPNET_TRY(launch_star_batch(pc, b.R, b.k, b.W, done, side));
    SPNET_CUDA_TRY(cudaEventRecord(b.ev_join, side));
  } else {
    SPNET_TRY(launch_star_batch(pc, b.R, b.k, b.W, done, s));
  }
  SPNET_TRY(launch_coarse_batch(pc, b.EP, b.k, b.ZC, b.cpart, done, s));
  if (side) SPNET_CUDA_TRY(cudaStreamWaitEvent(s, b.ev_join, 0));
  launch_bcombine(pc, b, 1, s);
  return SPNET_OK;
}

constexpr int BCHUNK = 8;  // iterations per replay of the captured graph

// z_j = B r_j (which 0), the coarse term only (1) or the star term only (2)
// for k <= 32 right-hand sides at once; r, z: device [k][n_free] in free order
int pc_apply_batch_free(spnet_pc_s* pc, int k, const double* r, double* z, int which) {
  cudaStream_t s = pc->op->stream;
  const int64_t N = pc->N;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  Batch b;
  SPNET_TRY(batch_alloc(pc, b, k, tmp, false));
  if (N == 0) return SPNET_OK;
  note_launch();
  k_cols_to_pc<<<pc->G, 256, 0, s>>>(N, k, pc->perm, r, b.R);
  const int wc = which != 2, ws = which != 1;
  launch_bupdate(pc, b, 1, s);
  if (wc) SPNET_TRY(launch_coarse_batch(pc, b.EP, b.k, b.ZC, b.cpart, nullptr, s));
  if (ws) SPNET_TRY(launch_star_batch(pc, b.R, b.k, b.W, nullptr, s));
  launch_bcombine(pc, b, 0, s, wc, ws);
  note_launch();
  k_cols_from_pc<<<pc->G, 256, 0, s>>>(N, k, pc->perm, b.Z, z);
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  SPNET_CUDA_TRY(cudaGetLastError());
  return SPNET_OK;
}

// k right-hand sides at once.  df, dg, dx: device arrays [k][n_dof], [k][n_dir],
// [k][n_dof] (x: the initial guess on entry if use_x0, u_hat on exit).  Fills
// stats[k].  A right-hand side whose recomputed residual misses rtol is
// finished on the one-right-hand-side path from where the batch left it.
int pcg_batch_run(spnet_op_s* op, spnet_pc_s* pc, int k, const double* df, const double* dg, double* dx,
                  int use_x0, double rtol, int maxit, spnet_stats* stats) {
  cudaStream_t s = op->stream;
  const int64_t N = pc->N, nd = op->n_dof, ndir = op->n_dir;
  const int G = pc->G;
  DevArena tmp;
  tmp.stream = s;
  Batch b;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  struct Guard {
    DevArena& a;
    Batch& b;
    cudaGraphExec_t& exec;
    cudaEvent_t &e0, &e1;
    ~Guard() {
      if (exec) cudaGraphExecDestroy(exec);
      if (b.ev_fork) cudaEventDestroy(b.ev_fork);
      if (b.ev_join) cudaEventDestroy(b.ev_join);
      if (b.side) cudaStreamDestroy(b.side);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      a.free_all();
    }
  } guard{tmp, b, exec, e0, e1};
  SPNET_TRY(batch_alloc(pc, b, k, tmp, true));
  SPNET_CUDA_TRY(cudaMemsetAsync(b.P, 0, sizeof(double) * N * k, s));
  SPNET_CUDA_TRY(cudaMemsetAsync(b.Q, 0, sizeof(double) * N * k, s));
  SPNET_CUDA_TRY(cudaMemsetAsync(b.Z, 0, sizeof(double) * N * k, s));
  SPNET_CUDA_TRY(cudaEventCreate(&e0));
  SPNET_CUDA_TRY(cudaEventCreate(&e1));
  SPNET_CUDA_TRY(cudaEventRecord(e0, s));
  // per right-hand side with the one-vector kernels: b_j, |b_j|^2, x_j, r_j = b_j - A x_j
  BScal h{};
  h.rtol = rtol;
  h.k = k;
  h.maxit = maxit;
  unsigned* cnt3 = &pc->scal->cnt[3];
  for (int j = 0; j < k; ++j) {
    note_launch();
    k_build_rhs<<<G, 256, 0, s>>>(N, pc->perm, op->free_dofs, df + (int64_t)j * nd, op->fd.ptr, op->fd.col,
                                  op->fd.val, dg + (int64_t)j * ndir, pc->b);
    note_launch();
    k_residual<<<G, 256, 0, s>>>(N, pc->b, nullptr, nullptr, pc->partial, &pc->scal->bb, cnt3);
    if (use_x0) {
      note_launch();
      k_x0_from_dofs<<<G, 256, 0, s>>>(N, pc->perm, op->free_dofs, dx + (int64_t)j * nd, pc->x);
      launch_spmv(pc->K, pc->x, pc->q, nullptr, G, pc->spmv_lanes, nullptr, s);
    } else {
      SPNET_CUDA_TRY(cudaMemsetAsync(pc->x, 0, sizeof(double) * N, s));
      SPNET_CUDA_TRY(cudaMemsetAsync(pc->q, 0, sizeof(double) * N, s));
    }
    note_launch();
    k_residual<<<G, 256, 0, s>>>(N, pc->b, pc->q, pc->r, pc->partial, &pc->scal->rr, cnt3);
    note_launch();
    k_col_put<<<G, 256, 0, s>>>(N, k, j, pc->x, b.X);
    note_launch();
    k_col_put<<<G, 256, 0, s>>>(N, k, j, pc->r, b.R);
    Scal sc{};
    SPNET_CUDA_TRY(cudaMemcpyAsync(&sc, pc->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s));
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));
    if (!std::isfinite(sc.bb) || !std::isfinite(sc.rr)) {  // (the guard releases the events)
      return fail(SPNET_ERR_BAD_INPUT, std::isfinite(sc.bb)
                                           ? "pcg_solve: non-finite initial guess"
                                           : "pcg_solve: non-finite right-hand side or Dirichlet data");
    }
    h.bb[j] = sc.bb;
    h.rr[j] = sc.rr;
    h.done[j] = (sc.bb == 0.0 || sqrt(sc.rr) <= rtol * sqrt(sc.bb) || maxit <= 0) ? 1 : 0;
  }
  int all = 1;
  for (int j = 0; j < k; ++j) all &= h.done[j];
  h.all_done = all;
  SPNET_CUDA_TRY(cudaMemcpyAsync(b.bs, &h, sizeof(BScal), cudaMemcpyHostToDevice, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  if (!all) {
    SPNET_TRY(precond_batch(pc, b, s));
    int graph_launches = 0;
    if (!profiling_on()) {
      SPNET_CUDA_TRY(cudaStreamCreateWithFlags(&b.side, cudaStreamNonBlocking));
      SPNET_CUDA_TRY(cudaEventCreateWithFlags(&b.ev_fork, cudaEventDisableTiming));
      SPNET_CUDA_TRY(cudaEventCreateWithFlags(&b.ev_join, cudaEventDisableTiming));
      cudaGraph_t g = nullptr;
      SPNET_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const long long before = launch_count();
      int rc = SPNET_OK;
      for (int it = 0; it < BCHUNK && rc == SPNET_OK; ++it) rc = batch_iteration(pc, b, s, b.side);
      graph_launches = (int)(launch_count() - before);
      add_launches(-graph_launches);
      cudaError_t e = cudaStreamEndCapture(s, &g);
      if (rc != SPNET_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return fail(SPNET_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        exec = nullptr;
        return fail(SPNET_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
    }
    for (;;) {
      if (exec) {
        add_launches(graph_launches);
        SPNET_CUDA_TRY(cudaGraphLaunch(exec, s));
      } else {
        for (int it = 0; it < BCHUNK; ++it) SPNET_TRY(batch_iteration(pc, b, s, nullptr));
      }
      SPNET_CUDA_TRY(cudaMemcpyAsync(&h, b.bs, sizeof(BScal), cudaMemcpyDeviceToHost, s));
      SPNET_CUDA_TRY(cudaStreamSynchronize(s));
      if (h.all_done) break;
    }
  }
  SPNET_CUDA_TRY(cudaEventRecord(e1, s));
  SPNET_CUDA_TRY(cudaEventSynchronize(e1));
  const double batch_ms = elapsed_ms(e0, e1);
  // per right-hand side: the solution, its residual recomputed in FP64, u_hat
  int worst = SPNET_OK;
  for (int j = 0; j < k; ++j) {
    double* xj = dx + (int64_t)j * nd;
    note_launch();
    k_col_get<<<G, 256, 0, s>>>(N, k, j, b.X, pc->x);
    if (h.bb[j] == 0.0) SPNET_CUDA_TRY(cudaMemsetAsync(pc->x, 0, sizeof(double) * N, s));
    note_launch();
    k_build_rhs<<<G, 256, 0, s>>>(N, pc->perm, op->free_dofs, df + (int64_t)j * nd, op->fd.ptr, op->fd.col,
                                  op->fd.val, dg + (int64_t)j * ndir, pc->b);
    launch_spmv(pc->K, pc->x, pc->q, nullptr, G, pc->spmv_lanes, nullptr, s);
    note_launch();
    k_residual<<<G, 256, 0, s>>>(N, pc->b, pc->q, pc->vtmp, pc->partial, &pc->scal->rr_true, cnt3);
    note_launch();
    k_expand<<<G, 256, 0, s>>>(nd, op->free_of, pc->iperm, pc->x, dg + (int64_t)j * ndir, xj);
    Scal sc{};
    SPNET_CUDA_TRY(cudaMemcpyAsync(&sc, pc->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s));
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));
    const double rel = h.bb[j] > 0.0 ? sqrt(sc.rr_true) / sqrt(h.bb[j]) : 0.0;
    spnet_stats st{};
    st.iterations = h.iters[j];
    st.relres = rel;
    st.relres_recursive = h.bb[j] > 0.0 ? sqrt(h.rr[j]) / sqrt(h.bb[j]) : 0.0;
    st.solve_ms = batch_ms;
    if (h.bb[j] == 0.0 || rel <= rtol) {
      st.converged = 1;
      st.status = SPNET_OK;
    } else if (h.iters[j] >= maxit) {
      st.status = SPNET_ERR_NO_CONVERGENCE;
      worst = SPNET_ERR_NO_CONVERGENCE;
    } else {  // finish this one alone, from where the batch left it
      spnet_stats one{};
      const int rc = pcg_run(op, pc, 1, df + (int64_t)j * nd, dg + (int64_t)j * ndir, xj, 1, rtol,
                             maxit - h.iters[j], SPNET_MEM_DEVICE, &one);
      if (rc != SPNET_OK && rc != SPNET_ERR_NO_CONVERGENCE) return rc;
      st.iterations += one.iterations;
      st.restarts = one.restarts + 1;
      st.relres = one.relres;
      st.relres_recursive = one.relres_recursive;
      st.converged = one.converged;
      st.status = one.status;
      if (!one.converged) worst = SPNET_ERR_NO_CONVERGENCE;
    }
    if (stats) stats[j] = st;
  }
  SPNET_CUDA_TRY(cudaGetLastError());
  return worst;
}

}  // namespace spnet
