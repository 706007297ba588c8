// The coarse solve z_c = A_0^{-1} r_c of P_0 (Section 4.1, eq. defPj).
//
// A_0 (m0 x m0, SPD) is inverted once at set-up by block Gauss-Jordan sweeps
// (pivot blocks of 64): sweeping pivot block K maps
//   A_ij -> A_ij - A_iK P A_Kj,  A_iK -> A_iK P,  A_Kj -> P A_Kj,  A_KK -> -P
// with P = A_KK^{-1}; after sweeping every block the matrix holds -A^{-1}.
// For an SPD matrix the pivot blocks are Schur complements, hence SPD, so no
// pivoting is needed.  Each application is then one dense symmetric
// matrix-vector product that every SM can share, instead of two dependent
// triangular solves.
// The sweeps and the product run in FP64 or, for the mixed-precision
// preconditioner, in FP32.
#include <climits>
#include <cmath>

#include "spnet_internal.cuh"

namespace spnet {

constexpr int NB = 64;  // pivot block

// invert the SPD pivot block D = Z[k0.., k0..] (kb x kb) into P by scalar sweeps
// in the arithmetic of T.  256 threads, each holding a 4 x 4 tile of D in
// registers (thread (tr, tc) owns rows 4tr.., columns 4tc..); row and column p
// of each step pass through shared memory, double-buffered so that one barrier
// per step suffices.  Every thread forms 1 / D_pp itself.
template <class T>
__global__ void __launch_bounds__(256) k_pivot_inverse(T* Z, int64_t ld, int k0, int kb, T* P, int* flags) {
  __shared__ T rowp[2][NB], colp[2][NB];
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  T d[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = 4 * tr + a, j = 4 * tc + b;
      d[a][b] = (i < kb && j < kb) ? Z[(int64_t)(k0 + i) * ld + (k0 + j)] : (T)0;
    }
  bool bad = false;
  for (int q = 0; q < NB / 4; ++q) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int p = 4 * q + a;
      if (p >= kb) break;  // uniform
      const int buf = p & 1;
      if (tr == q) {
#pragma unroll
        for (int b = 0; b < 4; ++b) rowp[buf][4 * tc + b] = d[a][b];
      }
      if (tc == q) {
#pragma unroll
        for (int b = 0; b < 4; ++b) colp[buf][4 * tr + b] = d[b][a];
      }
      __syncthreads();
      T piv = colp[buf][p];
      if (!(piv > (T)0)) {
        bad = true;
        piv = (T)1;
      }
      const T ip = (T)1 / piv;
      T cv[4], rv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cv[u] = colp[buf][4 * tr + u];
        rv[u] = rowp[buf][4 * tc + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const bool ri = 4 * tr + u == p, cj = 4 * tc + v == p;
          if (!ri && !cj) d[u][v] -= cv[u] * rv[v] * ip;
          else if (ri && cj) d[u][v] = -ip;
          else if (ri) d[u][v] = rv[v] * ip;
          else d[u][v] = cv[u] * ip;
        }
    }
  }
  if (bad && threadIdx.x == 0) atomicOr(flags, FLAG_COARSE_SPD);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = 4 * tr + a, j = 4 * tc + b;
      P[i * NB + j] = (i < kb && j < kb) ? -d[a][b] : (T)0;
    }
}

// R = Z[k0:k0+kb, :] (copy of the pivot rows), Tm = P R.  A block takes 16
// columns; thread (g, c) loads column c's kb pivot-row entries and forms rows
// 4g..4g+3 of P R for it.
template <class T>
__global__ void __launch_bounds__(256) k_panel(const T* Z, int64_t m0, int64_t ld, int k0, int kb,
                                               const T* P, T* R, T* Tm) {
  __shared__ T sP[NB][NB + 1];
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) sP[q / NB][q % NB] = P[q];
  __syncthreads();
  const int g = threadIdx.x >> 4;
  const int64_t c = (int64_t)blockIdx.x * 16 + (threadIdx.x & 15);
  if (c >= m0) return;
  T col[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) col[t] = t < kb ? Z[(int64_t)(k0 + t) * ld + c] : (T)0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int t = 4 * g + u;
    if (t < kb) R[(int64_t)t * m0 + c] = Z[(int64_t)(k0 + t) * ld + c];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int t = 4 * g + u;
    T acc = 0;
#pragma unroll
    for (int v = 0; v < NB; ++v) acc += sP[t][v] * col[v];
    if (t < kb) Tm[(int64_t)t * m0 + c] = acc;
  }
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::);
}

// the rank-kb sweep update: tiles of TB x TB entries, (TB/16)^2 per thread; only
// tiles on or above the block diagonal are computed, each writes itself and its
// mirror image (the swept matrix stays symmetric).  The tile's old values are
// copied to shared memory asynchronously while the update is computed.
template <class T, int TB>
__global__ void __launch_bounds__(256) k_sweep(T* Z, int64_t m0, int64_t ld, int k0, int kb, const T* P,
                                               const T* __restrict__ R, const T* __restrict__ Tm) {
  constexpr int RT = TB / 16;       // register tile
  constexpr int SO = TB + 16 / sizeof(T);  // padded row of the staged tile (16-byte aligned)
  extern __shared__ __align__(16) char sm_raw[];
  T (*sR)[TB] = reinterpret_cast<T (*)[TB]>(sm_raw);
  T (*sT)[TB] = reinterpret_cast<T (*)[TB]>(sm_raw + sizeof(T) * NB * TB);
  T (*sO)[SO] = reinterpret_cast<T (*)[SO]>(sm_raw + 2 * sizeof(T) * NB * TB);
  // map the linear block index to an upper-triangular tile (bi <= bj)
  const int nt = (int)((m0 + TB - 1) / TB);
  int rem = blockIdx.x, bi = 0;
  while (rem >= nt - bi) {
    rem -= nt - bi;
    ++bi;
  }
  const int bj = bi + rem;
  const int64_t i0 = (int64_t)bi * TB, j0 = (int64_t)bj * TB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  // old tile values -> sO (16-byte chunks; rows are 16-byte aligned, ld padded)
  constexpr int CH = TB * sizeof(T) / 16;  // chunks per tile row
  for (int q = threadIdx.x; q < TB * CH; q += 256) {
    const int li = q / CH, ch = q % CH;
    const int64_t i = i0 + li, j = j0 + ch * (16 / sizeof(T));
    if (i < m0 && j < ld) cp_async16(&sO[li][ch * (16 / sizeof(T))], &Z[i * ld + j]);
  }
  for (int q = threadIdx.x; q < NB * TB; q += 256) {
    const int t = q / TB, c = q % TB;
    sR[t][c] = (t < kb && i0 + c < m0) ? R[(int64_t)t * m0 + i0 + c] : (T)0;
    sT[t][c] = (t < kb && j0 + c < m0) ? Tm[(int64_t)t * m0 + j0 + c] : (T)0;
  }
  __syncthreads();
  T acc[RT][RT];
#pragma unroll
  for (int a = 0; a < RT; ++a)
#pragma unroll
    for (int b = 0; b < RT; ++b) acc[a][b] = 0;
  for (int t = 0; t < kb; ++t) {
    T ri[RT], tj[RT];
#pragma unroll
    for (int a = 0; a < RT; ++a) ri[a] = sR[t][ty + 16 * a];
#pragma unroll
    for (int b = 0; b < RT; ++b) tj[b] = sT[t][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
      for (int b = 0; b < RT; ++b) acc[a][b] += ri[a] * tj[b];
  }
  cp_async_wait_all();
  __syncthreads();
  // new values of the tile (i, j), in place in shared memory
#pragma unroll
  for (int a = 0; a < RT; ++a) {
    const int li = ty + 16 * a;
    const int64_t i = i0 + li;
    const bool iK = i >= k0 && i < k0 + kb;
#pragma unroll
    for (int b = 0; b < RT; ++b) {
      const int lj = tx + 16 * b;
      const int64_t j = j0 + lj;
      T v = 0;
      if (i < m0 && j < m0) {
        const bool jK = j >= k0 && j < k0 + kb;
        if (!iK && !jK) v = sO[li][lj] - acc[a][b];
        else if (iK && jK) v = -P[(i - k0) * NB + (j - k0)];
        else if (iK) v = sT[i - k0][lj];
        else v = Tm[(j - k0) * m0 + i];  // A_iK P = (P A_Ki)^T by symmetry
      }
      acc[a][b] = v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < RT; ++a)
#pragma unroll
    for (int b = 0; b < RT; ++b) sO[ty + 16 * a][tx + 16 * b] = acc[a][b];
  __syncthreads();
  for (int q = threadIdx.x; q < TB * TB; q += 256) {
    const int li = q / TB, lj = q % TB;
    const int64_t i = i0 + li, j = j0 + lj;
    if (i < m0 && j < m0) Z[i * ld + j] = sO[li][lj];
  }
  if (bi != bj) {
    for (int q = threadIdx.x; q < TB * TB; q += 256) {
      const int lj = q / TB, li = q % TB;  // write the mirror tile row by row
      const int64_t i = i0 + li, j = j0 + lj;
      if (i < m0 && j < m0) Z[j * ld + i] = sO[li][lj];
    }
  }
}

// mode 0: Z = A0 (rows padded to ld with zeros); mode 1: Z = -Z
template <class T>
__global__ void k_negate_from(const double* A0, T* Z, int64_t m0, int64_t ld, int mode) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m0 * ld;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / ld, j = q % ld;
    if (mode == 0) Z[q] = j < m0 ? (T)A0[i * m0 + j] : (T)0;
    else Z[q] = -Z[q];
  }
}

template <class T>
static int invert_impl(spnet_pc_s* pc, const double* A0) {
  cudaStream_t s = pc->op->stream;
  const int64_t m0 = pc->m0;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  // rows padded to 16 bytes so that the coarse product can load them as vectors
  const int64_t ld = (m0 + (16 / (int64_t)sizeof(T)) - 1) / (16 / (int64_t)sizeof(T)) * (16 / (int64_t)sizeof(T));
  T* Z = nullptr;
  SPNET_TRY(pc->mem.get(&Z, m0 * ld));
  pc->Z = Z;
  pc->ldz = ld;
  T *P = nullptr, *R = nullptr, *Tm = nullptr;
  SPNET_TRY(tmp.get(&P, NB * NB));
  SPNET_TRY(tmp.get(&R, NB * m0));
  SPNET_TRY(tmp.get(&Tm, NB * m0));
  const int grid = 4 * num_sms();
  note_launch();
  k_negate_from<T><<<grid, 256, 0, s>>>(A0, Z, m0, ld, 0);
  SPNET_CUDA_TRY(cudaMemsetAsync(pc->op->dflags, 0, sizeof(int), s));
  constexpr int TB = sizeof(T) == 4 ? 128 : 64;
  const int nt = (int)((m0 + TB - 1) / TB);
  const unsigned tiles = (unsigned)(nt * (nt + 1) / 2);
  const size_t smem = sizeof(T) * (2 * NB * TB + TB * (TB + 16 / sizeof(T)));
  static bool attr_set[64] = {};  // per device and instantiation; the size depends only on T
  int dev = 0;
  SPNET_CUDA_TRY(cudaGetDevice(&dev));
  dev &= 63;
  if (!attr_set[dev]) {
    SPNET_CUDA_TRY(cudaFuncSetAttribute(k_sweep<T, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set[dev] = true;
  }
  for (int k0 = 0; k0 < m0; k0 += NB) {
    const int kb = (int)((m0 - k0) < NB ? (m0 - k0) : NB);
    note_launch();
    k_pivot_inverse<T><<<1, 256, 0, s>>>(Z, ld, k0, kb, P, pc->op->dflags);
    note_launch();
    k_panel<T><<<(unsigned)((m0 + 15) / 16), 256, 0, s>>>(Z, m0, ld, k0, kb, P, R, Tm);
    note_launch();
    ProfScope ps(KID_SWEEP, s);
    k_sweep<T, TB><<<tiles, 256, smem, s>>>(Z, m0, ld, k0, kb, P, R, Tm);
  }
  note_launch();
  k_negate_from<T><<<grid, 256, 0, s>>>(A0, Z, m0, ld, 1);
  SPNET_CUDA_TRY(cudaGetLastError());
  return check_flags(pc->op->dflags, s, "setup_preconditioner (coarse matrix)");
}

int pc_coarse_invert(spnet_pc_s* pc, double* A0) {
  if (pc->m0 == 0) return SPNET_OK;
  if (pc->precision == SPNET_PREC_FP64) return invert_impl<double>(pc, A0);
  return invert_impl<float>(pc, A0);
}

// ---------------------------------------------------------------------------
// z_c = Z r_c with Z = A_0^{-1} symmetric: only the upper tiles (I <= J) of
// CT x CT are kept, packed tile after tile (row-major inside a tile, zero
// padded past m0), which halves the bytes of every application.  One block per
// stored tile reads it once and uses it twice:
//   row sums     Z_IJ r_J   -> part[I][J]   (the contribution of column block J to z_I)
//   column sums  Z_IJ^T r_I -> part[J][I]   (I < J: the contribution of row block I to z_J)
// Every part[R][K] has one writer.  A counter per row block R counts the parts
// written; the block that writes the last one sums part[R][0..nt-1] in K order
// (deterministic) into z_c and resets the counter for the next application.
// ---------------------------------------------------------------------------
constexpr int CT = 128;

__host__ __device__ inline int64_t n_upper_tiles(int nt) { return (int64_t)nt * (nt + 1) / 2; }

// linear upper-tile index -> (I, J), row-major over I <= J
__device__ inline void upper_tile(int t, int nt, int* I, int* J) {
  int i = 0;
  while (t >= nt - i) {
    t -= nt - i;
    ++i;
  }
  *I = i;
  *J = i + t;
}

template <class T>
__global__ void k_pack_tiles(const T* __restrict__ Z, int64_t m0, int64_t ld, int nt, T* __restrict__ tiles) {
  int I, J;
  upper_tile(blockIdx.x, nt, &I, &J);
  T* out = tiles + (int64_t)blockIdx.x * CT * CT;
  for (int q = threadIdx.x; q < CT * CT; q += blockDim.x) {
    const int64_t i = (int64_t)I * CT + q / CT, j = (int64_t)J * CT + q % CT;
    out[q] = (i < m0 && j < m0) ? Z[i * ld + j] : (T)0;
  }
}

template <class T>
struct Vec4 {
  T v[4];
};

__device__ __forceinline__ Vec4<float> load4(const float* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  return Vec4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Vec4<double> load4(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return Vec4<double>{{a.x, a.y, b.x, b.y}};
}

// r_c[ci] = (R_0 r)[ci] from the element corner sums E[e][c][a] around the mesh
// node of coarse dof ci (the restriction of Section 2.3): rtab[ci][cp] is the
// offset of E[e][c][a] for the element e at position cp around the node, -1
// where there is none; the same terms in the same order as the stand-alone
// restriction
__device__ __forceinline__ double restrict_one(int ci, const int32_t* __restrict__ rtab,
                                               const double* __restrict__ epart) {
  const int4 t0 = __ldg(reinterpret_cast<const int4*>(rtab + 8ll * ci));
  const int4 t1 = __ldg(reinterpret_cast<const int4*>(rtab + 8ll * ci) + 1);
  const int ix[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
  double v[8];
#pragma unroll
  for (int cp = 0; cp < 8; ++cp) v[cp] = ix[cp] >= 0 ? __ldg(&epart[ix[cp]]) : 0.0;
  double s = 0.0;
#pragma unroll
  for (int cp = 0; cp < 8; ++cp)
    if (ix[cp] >= 0) s += v[cp];
  return s;
}

// 256 threads: warp w takes tile rows [16w, 16w + 16), lane l columns [4l, 4l + 4).
// The input is r_c itself (rc != null) or, fused with the restriction, the
// element corner sums (rc == null).
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_coarse_symv(const T* __restrict__ tiles, int nt, int64_t m0,
                                                     const double* __restrict__ rc,
                                                     const double* __restrict__ epart,
                                                     const int32_t* __restrict__ rtab,
                                                     T* __restrict__ part,
                                                     unsigned* __restrict__ cnt, double* __restrict__ zc,
                                                     const int* done) {
  constexpr int RW = CT / 8;                  // rows per warp
  constexpr int RB = 8;                       // rows loaded per batch
  __shared__ T sI[CT], sJ[CT];
  __shared__ T scol[8][CT];
  __shared__ int red[2];
  if (done && *done) return;
  int I, J;
  upper_tile(blockIdx.x, nt, &I, &J);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* Zt = tiles + (int64_t)blockIdx.x * CT * CT + (int64_t)(wid * RW) * CT + 4 * lane;
  Vec4<T> v[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) v[k] = load4(Zt + (int64_t)k * CT);
  {
    const bool first = threadIdx.x < CT;
    const int64_t i = (int64_t)(first ? I : J) * CT + (threadIdx.x & (CT - 1));
    T val = (T)0;
    if (i < m0) val = (T)(rc ? rc[i] : restrict_one((int)i, rtab, epart));
    if (first) sI[threadIdx.x] = val;
    else sJ[threadIdx.x - CT] = val;
  }
  __syncthreads();
  T rj[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) rj[u] = sJ[4 * lane + u];
  T rowp[RW];
  T col[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int b = 0; b < RW; b += RB) {
    if (b > 0) {
#pragma unroll
      for (int k = 0; k < RB; ++k) v[k] = load4(Zt + (int64_t)(b + k) * CT);
    }
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      const T ri = sI[wid * RW + b + k];
      T acc = v[k].v[0] * rj[0];
#pragma unroll
      for (int u = 1; u < 4; ++u) acc += v[k].v[u] * rj[u];
      rowp[b + k] = acc;
#pragma unroll
      for (int u = 0; u < 4; ++u) col[u] += v[k].v[u] * ri;
    }
  }
  const T tot = reduce_scatter<RW>(rowp, lane);
  if (rs_writer<RW>(lane)) part[((int64_t)I * nt + J) * CT + wid * RW + rs_index<RW>(lane)] = tot;
  if (I != J) {
#pragma unroll
    for (int u = 0; u < 4; ++u) scol[wid][4 * lane + u] = col[u];
    __syncthreads();
    if (threadIdx.x < CT) {
      T sum = scol[0][threadIdx.x];
#pragma unroll
      for (int w = 1; w < 8; ++w) sum += scol[w][threadIdx.x];
      part[((int64_t)J * nt + I) * CT + threadIdx.x] = sum;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    red[0] = atomicAdd(&cnt[I], 1u) == (unsigned)(nt - 1) ? 1 : 0;
    red[1] = (I != J && atomicAdd(&cnt[J], 1u) == (unsigned)(nt - 1)) ? 1 : 0;
  }
  __syncthreads();
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if (!red[side]) continue;  // uniform over the block
    __threadfence();
    const int R = side == 0 ? I : J;
    if (threadIdx.x < CT) {
      const int64_t i = (int64_t)R * CT + threadIdx.x;
      const T* pr = part + (int64_t)R * nt * CT + threadIdx.x;
      double sum = 0.0;
      // eight independent loads in flight, summed in K order
      for (int K0 = 0; K0 < nt; K0 += 8) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = K0 + u < nt ? __ldcg(pr + (int64_t)(K0 + u) * CT) : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (K0 + u < nt) sum += (double)v[u];
      }
      if (i < m0) zc[i] = sum;
    }
    if (threadIdx.x == 0) cnt[R] = 0u;
  }
}

// z_c = A_0^{-1} r_c; with rc == null, r_c = R_0 r is formed from the element
// corner sums of the last update (restriction fused into the product)
void launch_coarse_apply(spnet_pc_s* pc, const double* rc, double* zc, const int* done,
                         cudaStream_t s) {
  if (pc->m0 == 0) return;
  const unsigned tiles = (unsigned)n_upper_tiles(pc->ctiles_n);
  note_launch();
  ProfScope ps(KID_COARSE, s);
  if (pc->precision == SPNET_PREC_FP64)
    k_coarse_symv<double><<<tiles, 256, 0, s>>>((const double*)pc->ctiles, pc->ctiles_n, pc->m0, rc, pc->epart,
                                                 pc->rtab, (double*)pc->cpart, pc->ccnt, zc, done);
  else
    k_coarse_symv<float><<<tiles, 256, 0, s>>>((const float*)pc->ctiles, pc->ctiles_n, pc->m0, rc, pc->epart,
                                                pc->rtab, (float*)pc->cpart, pc->ccnt, zc, done);
}

// rtab[ci][cp]: offset of the corner sum of the element at position cp around
// the mesh node of coarse dof ci (corner nc-1-cp of that element), -1 if none
__global__ void k_restrict_table(int64_t nmc, Mesh m, int ndof, const int32_t* __restrict__ cidx,
                                 int32_t* __restrict__ rtab) {
  for (int64_t ka = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ka < nmc; ka += (int64_t)gridDim.x * blockDim.x) {
    const int ci = cidx[ka];
    if (ci < 0) continue;
    const int k = (int)(ka / ndof), a = (int)(ka % ndof);
    int km[3];
    mesh_multi(m, k, km);
    for (int cp = 0; cp < 8; ++cp) {
      int off = -1;
      if (cp < m.nc) {
        const int e = elem_around(m, km, cp);
        if (e >= 0) off = (int)(((int64_t)e * m.nc + (m.nc - 1 - cp)) * ndof + a);
      }
      rtab[8ll * ci + cp] = off;
    }
  }
}

// pack the upper tiles of Z, release the full matrix, allocate the parts and counters
template <class T>
static int pack_coarse_tiles(spnet_pc_s* pc) {
  cudaStream_t s = pc->op->stream;
  const int nt = (int)((pc->m0 + CT - 1) / CT);
  const int64_t nti = n_upper_tiles(nt);
  T* tiles = nullptr;
  T* part = nullptr;
  SPNET_TRY(pc->mem.get(&tiles, nti * CT * CT));
  SPNET_TRY(pc->mem.get(&part, (int64_t)nt * nt * CT));
  SPNET_TRY(pc->mem.get(&pc->ccnt, nt));
  SPNET_CUDA_TRY(cudaMemsetAsync(pc->ccnt, 0, sizeof(unsigned) * nt, s));
  const int64_t nmc = (int64_t)pc->n_mesh * pc->ndof;
  if ((int64_t)pc->n_elem * pc->nc * pc->ndof > INT32_MAX)
    return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: too many element corner sums for 32-bit offsets");
  SPNET_TRY(pc->mem.get(&pc->rtab, 8ll * pc->m0));
  note_launch();
  k_restrict_table<<<(unsigned)((nmc + 255) / 256), 256, 0, s>>>(nmc, mesh_of_pc(pc), pc->ndof, pc->cidx, pc->rtab);
  note_launch();
  k_pack_tiles<T><<<(unsigned)nti, 256, 0, s>>>((const T*)pc->Z, pc->m0, pc->ldz, nt, tiles);
  SPNET_CUDA_TRY(cudaGetLastError());
  pc->mem.release(pc->Z);
  pc->Z = nullptr;
  pc->ctiles = tiles;
  pc->cpart = part;
  pc->ctiles_n = nt;
  return SPNET_OK;
}

int coarse_gemv_prepare(spnet_pc_s* pc) {
  if (pc->m0 == 0) return SPNET_OK;
  if (pc->precision == SPNET_PREC_FP64) return pack_coarse_tiles<double>(pc);
  return pack_coarse_tiles<float>(pc);
}

}  // namespace spnet
