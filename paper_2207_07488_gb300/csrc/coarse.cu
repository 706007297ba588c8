// The coarse solve z_c = A_0^{-1} r_c of P_0 (Section 4.1, eq. defPj).
//
// A_0 (m0 x m0, SPD) is inverted once at set-up by block Gauss-Jordan sweeps
// (pivot blocks of 64): sweeping pivot block K maps
//   A_ij -> A_ij - A_iK P A_Kj,  A_iK -> A_iK P,  A_Kj -> P A_Kj,  A_KK -> -P
// with P = A_KK^{-1}; after sweeping every block the matrix holds -A^{-1}.
// For an SPD matrix the pivot blocks are Schur complements, hence SPD, so no
// pivoting is needed.  Each application is then one dense matrix-vector
// product that every SM can share, instead of two dependent triangular solves.
// The sweeps and the product run in FP64 or, for the mixed-precision
// preconditioner, in FP32.
#include <cmath>

#include "spnet_internal.cuh"

namespace spnet {

constexpr int NB = 64;  // pivot block

// invert the SPD pivot block D = Z[k0.., k0..] (kb x kb) into P by scalar sweeps
// in the arithmetic of T; 1024 threads, 2 x 2 entries each
template <class T>
__global__ void __launch_bounds__(1024) k_pivot_inverse(T* Z, int64_t ld, int k0, int kb, T* P, int* flags) {
  __shared__ T D[NB][NB + 1];
  __shared__ T col[NB], row[NB];
  __shared__ T ipiv;
  const int tj = threadIdx.x, ti = threadIdx.y;  // 32 x 32
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = ti + 32 * a, j = tj + 32 * b;
      D[i][j] = (i < kb && j < kb) ? Z[(int64_t)(k0 + i) * ld + (k0 + j)] : (T)0;
    }
  __syncthreads();
  for (int p = 0; p < kb; ++p) {
    if (ti == 0 && tj == 0) {
      T piv = D[p][p];
      if (!(piv > (T)0)) {
        atomicOr(flags, FLAG_COARSE_SPD);
        piv = (T)1;
      }
      ipiv = (T)1 / piv;
    }
    if (ti == 0) {
      row[tj] = D[p][tj];
      row[tj + 32] = D[p][tj + 32];
    }
    if (tj == 0) {
      col[ti] = D[ti][p];
      col[ti + 32] = D[ti + 32][p];
    }
    __syncthreads();
    const T ip = ipiv;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const int i = ti + 32 * a, j = tj + 32 * b;
        if (i < kb && j < kb) {
          if (i != p && j != p) D[i][j] -= col[i] * row[j] * ip;
          else if (i == p && j == p) D[i][j] = -ip;
          else if (i == p) D[i][j] = row[j] * ip;
          else D[i][j] = col[i] * ip;
        }
      }
    __syncthreads();
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = ti + 32 * a, j = tj + 32 * b;
      P[i * NB + j] = (i < kb && j < kb) ? -D[i][j] : (T)0;
    }
}

// R = Z[k0:k0+kb, :] (copy of the pivot rows), Tm = P R
template <class T>
__global__ void __launch_bounds__(128) k_panel(const T* Z, int64_t m0, int64_t ld, int k0, int kb,
                                               const T* P, T* R, T* Tm) {
  __shared__ T sP[NB][NB];
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) sP[q / NB][q % NB] = P[q];
  __syncthreads();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < m0;
       c += (int64_t)gridDim.x * blockDim.x) {
    T col[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) col[t] = t < kb ? Z[(int64_t)(k0 + t) * ld + c] : (T)0;
#pragma unroll
    for (int t = 0; t < NB; ++t)
      if (t < kb) R[(int64_t)t * m0 + c] = col[t];
    for (int t = 0; t < kb; ++t) {
      T acc = 0;
#pragma unroll
      for (int u = 0; u < NB; ++u) acc += sP[t][u] * col[u];
      Tm[(int64_t)t * m0 + c] = acc;
    }
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
    k_pivot_inverse<T><<<1, dim3(32, 32), 0, s>>>(Z, ld, k0, kb, P, pc->op->dflags);
    note_launch();
    k_panel<T><<<(unsigned)((m0 + 127) / 128), 128, 0, s>>>(Z, m0, ld, k0, kb, P, R, Tm);
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

// z_c = Z r_c: r_c staged in shared memory, one warp per row, 16-byte loads of Z
template <class T, class V>
__global__ void __launch_bounds__(256) k_coarse_gemv(const T* __restrict__ Z, int64_t m0, int64_t ld,
                                                     const double* __restrict__ rc,
                                                     double* __restrict__ zc, const int* done) {
  extern __shared__ __align__(16) char sm_raw[];
  T* srv = reinterpret_cast<T*>(sm_raw);
  if (done && *done) return;
  for (int64_t c = threadIdx.x; c < ld; c += blockDim.x) srv[c] = c < m0 ? (T)rc[c] : (T)0;
  __syncthreads();
  constexpr int VW = sizeof(V) / sizeof(T);
  const int lane = threadIdx.x & 31;
  const int64_t nv = ld / VW;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < m0; row += nw) {
    const V* zr = reinterpret_cast<const V*>(Z + row * ld);
    T acc = 0;
#pragma unroll 4
    for (int64_t c = lane; c < nv; c += 32) {
      const V z = __ldg(&zr[c]);
      const T* zz = reinterpret_cast<const T*>(&z);
#pragma unroll
      for (int u = 0; u < VW; ++u) acc += zz[u] * srv[c * VW + u];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) zc[row] = (double)acc;
  }
}

void launch_coarse_apply(spnet_pc_s* pc, const double* rc, double* zc, const int* done,
                         cudaStream_t s) {
  if (pc->m0 == 0) return;
  int blocks = 2 * num_sms();
  const int64_t rows_blocks = (pc->m0 + 7) / 8;
  if (blocks > rows_blocks) blocks = (int)rows_blocks;
  const size_t vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  const size_t smem = vb * (size_t)pc->ldz;
  note_launch();
  ProfScope ps(KID_COARSE, s);
  if (pc->precision == SPNET_PREC_FP64)
    k_coarse_gemv<double, double2><<<blocks, 256, smem, s>>>((const double*)pc->Z, pc->m0, pc->ldz, rc, zc, done);
  else
    k_coarse_gemv<float, float4><<<blocks, 256, smem, s>>>((const float*)pc->Z, pc->m0, pc->ldz, rc, zc, done);
}

int coarse_gemv_prepare(spnet_pc_s* pc) {
  if (pc->m0 == 0) return SPNET_OK;
  const size_t vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  const size_t smem = vb * (size_t)pc->ldz;
  if (smem > 220 * 1024)
    return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: coarse space too large for the staged product");
  if (smem > 48 * 1024) {
    if (pc->precision == SPNET_PREC_FP64)
      SPNET_CUDA_TRY(cudaFuncSetAttribute(k_coarse_gemv<double, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else
      SPNET_CUDA_TRY(cudaFuncSetAttribute(k_coarse_gemv<float, float4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  return SPNET_OK;
}

}  // namespace spnet
