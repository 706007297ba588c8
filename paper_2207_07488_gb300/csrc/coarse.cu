// The coarse solve z_c = A_0^{-1} r_c of P_0 (Section 4.1, eq. defPj).
//
// A_0 (m0 x m0, SPD) is inverted once at set-up by block Gauss-Jordan sweeps
// (pivot blocks of 64): sweeping pivot block K maps
//   A_ij -> A_ij - A_iK P A_Kj,  A_iK -> A_iK P,  A_Kj -> P A_Kj,  A_KK -> -P
// with P = A_KK^{-1}; after sweeping every block the matrix holds -A^{-1}.
// For an SPD matrix the pivot blocks are Schur complements, hence SPD, so no
// pivoting is needed.
// A_0 is singular when the basis functions truncated to the free dofs are
// linearly dependent; P_0, the projection onto their span V_H, is still
// defined.  A scalar pivot d_k that is at most DROP64 = 1e-8 times the
// original diagonal entry A0_kk marks a function in the span of the ones swept
// before it (exact dependence leaves d_k at rounding level, ~1e-11 or less,
// while independent functions of the workloads keep 1e-6 or more): it is not
// swept, and its row and column of P are zeroed, so it never enters the other
// blocks.  A sweep over a set of pivots gives the inverse of the swept block
// whatever the order, so the result is A_KK^{-1} on the kept functions K and
// zero elsewhere: the same P_0.  FP32 sweeps cannot tell rounding from a small
// pivot once one small pivot is kept, so the mixed-precision set-up sweeps in
// FP32 only while every pivot stays above TRIG32 = 1e-3 of its diagonal entry
// (ordinary meshes: 0.4 and more); otherwise the inverse is formed in FP64,
// with the drops, and rounded to FP32.  Each application is then one dense symmetric
// matrix-vector product that every SM can share, instead of two dependent
// triangular solves.
// The sweeps and the product run in FP64 or, for the mixed-precision
// preconditioner, in FP32.
#include <climits>
#include <atomic>
#include <cmath>

#include "spnet_internal.cuh"

namespace spnet {

constexpr int NB = 64;   // pivot block, and the sub-tile a sweep block updates
constexpr int SP = NB + 8;  // row pitch of the sweep's shared R and Tm slices (conflict-free fragments)
constexpr int CT = 128;  // storage tile

// ---------------------------------------------------------------------------
// Storage.  Z is symmetric throughout the sweeps, so only its upper tiles
// (I <= J) of CT x CT entries are kept, packed tile after tile (row-major inside
// a tile, zero padded past m0); a diagonal tile holds both of its triangles.
// The coarse product reads the same array.
// ---------------------------------------------------------------------------
__host__ __device__ inline int64_t n_upper_tiles(int nt) { return (int64_t)nt * (nt + 1) / 2; }
__host__ __device__ inline int64_t tile_index(int I, int J, int nt) {
  return (int64_t)I * nt - (int64_t)I * (I - 1) / 2 + (J - I);
}

// linear index -> (I, J) of the upper triangle of an n x n grid, row-major
__device__ inline void upper_tile(int64_t t, int n, int* I, int* J) {
  int i = 0;
  while (t >= n - i) {
    t -= n - i;
    ++i;
  }
  *I = i;
  *J = i + (int)t;
}

// entry (i, j) of the symmetric Z, any i, j
template <class T>
__device__ inline T zat(const T* tiles, int nt, int64_t i, int64_t j) {
  if (i / CT > j / CT) {
    const int64_t t = i;
    i = j;
    j = t;
  }
  return tiles[tile_index((int)(i / CT), (int)(j / CT), nt) * CT * CT + (i % CT) * CT + (j % CT)];
}

// Invert the SPD block held 4 x 4 per thread by 256 threads (thread (tr, tc)
// owns rows 4tr.., columns 4tc.. of a 64 x 64 block; kb valid rows) by scalar
// Gauss-Jordan sweeps in the arithmetic of T: sweeping pivot p maps
// D_ij -> D_ij - D_ip D_pj / D_pp, D_ip -> D_ip / D_pp, D_pj -> D_pj / D_pp,
// D_pp -> -1 / D_pp; after kb pivots the block holds -D^{-1}.  Row and column
// p pass through shared memory, double-buffered (one barrier per pivot); every
// thread forms 1 / D_pp itself.  Returns true where a pivot was not positive.
constexpr double DROP64 = 1e-8;  // FP64 sweeps: relative pivot at or below which a function is dropped
constexpr double TRIG32 = 1e-3;  // FP32 sweeps: relative pivot at or below which FP64 takes over

// As above, with dropping: dg holds the original diagonal entries of the block's
// rows; a pivot at or below tol times its entry is not swept.  Returns the bitmask
// of the dropped pivots (uniform over the threads).
template <class T>
__device__ uint64_t invert_block_regs(T (&d)[4][4], int kb, T (*rowp)[NB], T (*colp)[NB], const double* dg,
                                      double tol) {
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  uint64_t dropped = 0;
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
      const T piv = colp[buf][p];
      if (!((double)piv > tol * dg[p])) {  // in the span of the pivots kept so far
        dropped |= 1ull << p;
        continue;
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
  return dropped;
}

// P = (the inverted block) = -(d after the sweeps), zero outside kb x kb and in the
// rows and columns of dropped pivots
template <class T>
__device__ void store_pivot(const T (&d)[4][4], int kb, uint64_t dropped, T* P) {
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = 4 * tr + a, j = 4 * tc + b;
      const bool off = ((dropped >> i) & 1) || ((dropped >> j) & 1);
      P[i * NB + j] = (i < kb && j < kb && !off) ? -d[a][b] : (T)0;
    }
}

// the upper tiles of A_0 (dense FP64, m0 x m0) in the arithmetic of T
template <class T>
__global__ void k_tiles_from_A0(const double* __restrict__ A0, int64_t m0, int nt, T* __restrict__ tiles) {
  int I, J;
  upper_tile(blockIdx.x, nt, &I, &J);
  T* out = tiles + (int64_t)blockIdx.x * CT * CT;
  for (int q = threadIdx.x; q < CT * CT; q += blockDim.x) {
    const int64_t i = (int64_t)I * CT + q / CT, j = (int64_t)J * CT + q % CT;
    out[q] = (i < m0 && j < m0) ? (T)A0[i * m0 + j] : (T)0;
  }
}

// the first pivot block (its inverse P); later ones are inverted by the sweep
template <class T>
__global__ void __launch_bounds__(256) k_pivot_inverse(const T* tiles, int nt, int k0, int kb, T* P,
                                                       const double* diag0, double tol, int* ndrop) {
  __shared__ T rowp[2][NB], colp[2][NB];
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  T d[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = 4 * tr + a, j = 4 * tc + b;
      d[a][b] = (i < kb && j < kb) ? zat(tiles, nt, k0 + i, k0 + j) : (T)0;
    }
  const uint64_t dropped = invert_block_regs(d, kb, rowp, colp, diag0 + k0, tol);
  if (threadIdx.x == 0 && dropped) atomicAdd(ndrop, __popcll(dropped));
  store_pivot(d, kb, dropped, P);
}

// Tm = P R with R the pivot rows Z[k0 + t][:] (rows of length ldr).  The first
// step reads them from the tiles and writes R (zero past m0 and past kb);
// later steps find R written by the previous sweep.  A block takes 16
// columns; thread (g, c) forms rows 4g..4g+3 of P R for column c.
template <class T>
__global__ void __launch_bounds__(256) k_panel(const T* __restrict__ tiles, int nt, int64_t m0, int64_t ldr, int k0,
                                               int kb, const T* __restrict__ P, T* __restrict__ R,
                                               T* __restrict__ Tm, int from_tiles) {
  __shared__ T sP[NB][NB + 1];
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) sP[q / NB][q % NB] = P[q];
  __syncthreads();
  const int g = threadIdx.x >> 4;
  const int64_t c = (int64_t)blockIdx.x * 16 + (threadIdx.x & 15);
  if (c >= ldr) return;
  T col[NB];
  if (from_tiles) {
#pragma unroll
    for (int t = 0; t < NB; ++t) col[t] = (t < kb && c < m0) ? zat(tiles, nt, k0 + t, c) : (T)0;
  } else {
#pragma unroll
    for (int t = 0; t < NB; ++t) col[t] = R[(int64_t)t * ldr + c];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int t = 4 * g + u;
    T acc = 0;
#pragma unroll
    for (int v = 0; v < NB; ++v) acc += sP[t][v] * col[v];
    if (from_tiles) R[(int64_t)t * ldr + c] = (t < kb && c < m0) ? zat(tiles, nt, k0 + t, c) : (T)0;
    Tm[(int64_t)t * ldr + c] = acc;
  }
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::);
}

// TF32 tensor-core products (mma.sync m16n8k8, FP32 accumulation) with each FP32 operand
// split in a high and a low TF32 part: x = hi + lo, hi = tf32(x), lo = tf32(x - hi)
__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_bits(x);
  lo = tf32_bits(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_m16n8k8_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <class T>
struct V4 {
  T v[4];
};
// four consecutive T (16-byte aligned; 32 for double)
template <class T>
__device__ __forceinline__ V4<T> ld4s(const T* p) {
  V4<T> r;
  if (sizeof(T) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    r.v[0] = a.x;
    r.v[1] = a.y;
    r.v[2] = a.z;
    r.v[3] = a.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *(reinterpret_cast<const double2*>(p) + 1);
    r.v[0] = a.x;
    r.v[1] = a.y;
    r.v[2] = b.x;
    r.v[3] = b.y;
  }
  return r;
}
template <class T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
  if (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *(reinterpret_cast<double2*>(p) + 1) = make_double2(v[2], v[3]);
  }
}

// One sweep (pivot sub-tile kp = k0 / 64 of a 64-grid with n64 sub-tiles per
// side): every sub-tile (a, b), a <= b, of the upper tiles, 64 x 64 per block,
// 4 x 4 per thread:
//   a, b != kp:        Z_ab -= R[:, a]^T Tm[:, b]       (= Z_aK P Z_Kb)
//   a == b == kp:      -P
//   a == kp:           Tm[:, b]                          (P Z_Kb)
//   b == kp:           Tm[:, a]^T                        (Z_aK P, by symmetry)
// The upper-right sub-tile of a diagonal storage tile also writes its
// transpose into the lower-left one.  The sub-tiles of row kp + 1 (and, as
// transposes, of column kp + 1) also write their new values into Rn, the
// pivot rows of the next step.  Block 0 updates the next pivot block
// (kp + 1, kp + 1) and then inverts it into Pn: the next step needs no
// separate pivot kernel, and its work hides behind the other blocks.
template <class T>
__global__ void __launch_bounds__(256) k_sweep(T* __restrict__ tiles, int nt, int n64, int64_t m0, int64_t ldr,
                                               int k0, const T* __restrict__ P, const T* __restrict__ R,
                                               const T* __restrict__ Tm, T* __restrict__ Pn, T* __restrict__ Rn,
                                               const double* __restrict__ diag0, double tol, int* ndrop) {
  extern __shared__ __align__(16) char sm_sweep[];  // R and Tm slices, NB rows of pitch SP each
  T (*sR)[SP] = reinterpret_cast<T (*)[SP]>(sm_sweep);
  T (*sT)[SP] = reinterpret_cast<T (*)[SP]>(sm_sweep + sizeof(T) * NB * SP);
  const int kp = k0 / NB;
  const bool has_next = (int64_t)(kp + 1) * NB < m0;
  // block -> sub-tile: block 0 takes the next pivot block, the rest go in order
  int64_t L = blockIdx.x;
  if (has_next) {
    const int64_t Lp = tile_index(kp + 1, kp + 1, n64);
    L = blockIdx.x == 0 ? Lp : ((int64_t)blockIdx.x <= Lp ? (int64_t)blockIdx.x - 1 : (int64_t)blockIdx.x);
  }
  int a, b;
  upper_tile(L, n64, &a, &b);
  const int64_t i0 = (int64_t)a * NB, j0 = (int64_t)b * NB;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  T* zt = tiles + tile_index(a >> 1, b >> 1, nt) * CT * CT + (a & 1) * NB * CT + (b & 1) * NB;
  // R and Tm slices -> shared memory (16-byte chunks; rows of length ldr, a multiple of 64)
  constexpr int CH = NB * (int)sizeof(T) / 16;  // chunks per row
  for (int q = threadIdx.x; q < NB * CH; q += 256) {
    const int t = q / CH, ch = q % CH;
    const int e = ch * (16 / (int)sizeof(T));
    cp_async16(&sR[t][e], R + (int64_t)t * ldr + i0 + e);
    cp_async16(&sT[t][e], Tm + (int64_t)t * ldr + j0 + e);
  }
  // old values
  T d[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const V4<T> o = ld4s(zt + (4 * ty + u) * CT + 4 * tx);
#pragma unroll
    for (int v = 0; v < 4; ++v) d[u][v] = o.v[v];
  }
  cp_async_wait_all();
  __syncthreads();
  const int kb = (int)((m0 - k0) < NB ? (m0 - k0) : NB);
  if (a != kp && b != kp) {
    if constexpr (sizeof(T) == 4) {
      // the rank-kb product on the tensor cores: warp w forms rows 16 (w % 4) .. +16 and
      // columns 32 (w / 4) .. +32 of sum_t R[t][i] Tm[t][j] as four 16 x 8 tiles, each
      // product as lo*hi + hi*lo + hi*hi of the split operands; then the products go
      // through shared memory (in place of the R slice) to the 4 x 4 layout of d
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, tq = lane & 3;
      const int ib = 16 * (w & 3), jb = 32 * (w >> 2);
      float c[4][4];
#pragma unroll
      for (int n8 = 0; n8 < 4; ++n8)
#pragma unroll
        for (int e = 0; e < 4; ++e) c[n8][e] = 0.f;
      for (int t0 = 0; t0 < kb; t0 += 8) {
        const bool k0ok = t0 + tq < kb, k1ok = t0 + tq + 4 < kb;
        uint32_t ah[4], al[4];
        tf32_split(k0ok ? (float)sR[t0 + tq][ib + g] : 0.f, ah[0], al[0]);
        tf32_split(k0ok ? (float)sR[t0 + tq][ib + g + 8] : 0.f, ah[1], al[1]);
        tf32_split(k1ok ? (float)sR[t0 + tq + 4][ib + g] : 0.f, ah[2], al[2]);
        tf32_split(k1ok ? (float)sR[t0 + tq + 4][ib + g + 8] : 0.f, ah[3], al[3]);
#pragma unroll
        for (int n8 = 0; n8 < 4; ++n8) {
          uint32_t bh0, bl0, bh1, bl1;
          tf32_split(k0ok ? (float)sT[t0 + tq][jb + 8 * n8 + g] : 0.f, bh0, bl0);
          tf32_split(k1ok ? (float)sT[t0 + tq + 4][jb + 8 * n8 + g] : 0.f, bh1, bl1);
          mma_m16n8k8_tf32(c[n8], al, bh0, bh1);
          mma_m16n8k8_tf32(c[n8], ah, bl0, bl1);
          mma_m16n8k8_tf32(c[n8], ah, bh0, bh1);
        }
      }
      __syncthreads();  // every warp is done with the slices
#pragma unroll
      for (int n8 = 0; n8 < 4; ++n8) {
        const int j = jb + 8 * n8 + 2 * tq;
        sR[ib + g][j] = c[n8][0];
        sR[ib + g][j + 1] = c[n8][1];
        sR[ib + g + 8][j] = c[n8][2];
        sR[ib + g + 8][j + 1] = c[n8][3];
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const V4<T> pr = ld4s(&sR[4 * ty + u][4 * tx]);
#pragma unroll
        for (int v = 0; v < 4; ++v) d[u][v] -= pr.v[v];
      }
    } else {
      T acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = (T)0;
      for (int t = 0; t < kb; ++t) {
        const V4<T> ri = ld4s(&sR[t][4 * ty]);
        const V4<T> tj = ld4s(&sT[t][4 * tx]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += ri.v[u] * tj.v[v];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) d[u][v] -= acc[u][v];
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int li = 4 * ty + u, lj = 4 * tx + v;
        if (a == kp && b == kp) d[u][v] = -P[li * NB + lj];
        else if (a == kp) d[u][v] = sT[li][lj];
        else d[u][v] = Tm[(int64_t)lj * ldr + i0 + li];
      }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) st4(zt + (4 * ty + u) * CT + 4 * tx, d[u]);
  if ((a & 1) == 0 && b == a + 1) {  // mirror into the lower-left sub-tile of the diagonal tile
    T* zl = tiles + tile_index(a >> 1, a >> 1, nt) * CT * CT + NB * CT;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const T col[4] = {d[0][v], d[1][v], d[2][v], d[3][v]};
      st4(zl + (4 * tx + v) * CT + 4 * ty, col);
    }
  }
  if (has_next && a == kp + 1) {  // pivot rows of the next step, row by row
#pragma unroll
    for (int u = 0; u < 4; ++u) st4(Rn + (int64_t)(4 * ty + u) * ldr + j0 + 4 * tx, d[u]);
  } else if (has_next && b == kp + 1) {  // ... and from the column above them, transposed
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const T col[4] = {d[0][v], d[1][v], d[2][v], d[3][v]};
      st4(Rn + (int64_t)(4 * tx + v) * ldr + i0 + 4 * ty, col);
    }
  }
  if (has_next && blockIdx.x == 0) {  // the next pivot block, already updated: invert it
    __shared__ T rowp[2][NB], colp[2][NB];
    const int kbn = (int)((m0 - k0 - NB) < NB ? (m0 - k0 - NB) : NB);
    const uint64_t dropped = invert_block_regs(d, kbn, rowp, colp, diag0 + k0 + NB, tol);
    if (threadIdx.x == 0 && dropped) atomicAdd(ndrop, __popcll(dropped));
    store_pivot(d, kbn, dropped, Pn);
  }
}

__global__ void k_diag_of(const double* __restrict__ A0, int64_t m0, double* __restrict__ dg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m0; i += (int64_t)gridDim.x * blockDim.x)
    dg[i] = A0[i * m0 + i];
}

template <class T>
__global__ void k_negate(T* z, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    z[q] = -z[q];
}

// Sweep the upper tiles of A_0 (T arithmetic) into the upper tiles of A_0^{-1}
// (on the kept functions); *ndrop receives the count of pivots at or below tol.
template <class T>
static int sweep_inverse(spnet_pc_s* pc, const double* A0, T* tiles, double tol, int* ndrop_out) {
  cudaStream_t s = pc->op->stream;
  const int64_t m0 = pc->m0;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const int nt = (int)((m0 + CT - 1) / CT);
  const int n64 = (int)((m0 + NB - 1) / NB);
  const int64_t ldr = (int64_t)n64 * NB;
  const int64_t nti = n_upper_tiles(nt);
  T *P = nullptr, *R = nullptr, *Tm = nullptr;
  SPNET_TRY(tmp.get(&P, 2 * NB * NB));
  SPNET_TRY(tmp.get(&R, 2 * NB * ldr));  // pivot rows of this step and of the next
  SPNET_TRY(tmp.get(&Tm, NB * ldr));
  SPNET_CUDA_TRY(cudaMemsetAsync(R, 0, sizeof(T) * 2 * NB * ldr, s));
  SPNET_CUDA_TRY(cudaMemsetAsync(Tm, 0, sizeof(T) * NB * ldr, s));
  double* diag0 = nullptr;  // original diagonal of A_0 (the drop test's scale), padded to ldr
  int* ndrop = nullptr;
  SPNET_TRY(tmp.get(&diag0, ldr));
  SPNET_TRY(tmp.get(&ndrop, 1));
  SPNET_CUDA_TRY(cudaMemsetAsync(diag0, 0, sizeof(double) * ldr, s));
  SPNET_CUDA_TRY(cudaMemsetAsync(ndrop, 0, sizeof(int), s));
  note_launch();
  k_diag_of<<<(unsigned)((m0 + 255) / 256), 256, 0, s>>>(A0, m0, diag0);
  note_launch();
  k_tiles_from_A0<T><<<(unsigned)nti, 256, 0, s>>>(A0, m0, nt, tiles);
  note_launch();
  k_pivot_inverse<T><<<1, 256, 0, s>>>(tiles, nt, 0, (int)(m0 < NB ? m0 : NB), P, diag0, tol, ndrop);
  const unsigned subtiles = (unsigned)n_upper_tiles(n64);
  const size_t sweep_smem = 2 * sizeof(T) * NB * SP;
  if (sweep_smem > 48 * 1024) {
    static std::atomic<bool> attr_set[64];  // per device; the size depends only on T
    int dev = 0;
    SPNET_CUDA_TRY(cudaGetDevice(&dev));
    dev &= 63;
    if (!attr_set[dev]) {
      SPNET_CUDA_TRY(cudaFuncSetAttribute(k_sweep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem));
      attr_set[dev] = true;
    }
  }
  for (int k0 = 0, step = 0; k0 < m0; k0 += NB, ++step) {
    const int kb = (int)((m0 - k0) < NB ? (m0 - k0) : NB);
    T* Pc = P + (step & 1) * NB * NB;
    T* Pn = P + ((step + 1) & 1) * NB * NB;
    T* Rc = R + (step & 1) * NB * ldr;
    T* Rn = R + ((step + 1) & 1) * NB * ldr;
    note_launch();
    k_panel<T><<<(unsigned)(ldr / 16), 256, 0, s>>>(tiles, nt, m0, ldr, k0, kb, Pc, Rc, Tm, step == 0 ? 1 : 0);
    note_launch();
    ProfScope ps(KID_SWEEP, s);
    k_sweep<T><<<subtiles, 256, sweep_smem, s>>>(tiles, nt, n64, m0, ldr, k0, Pc, Rc, Tm, Pn, Rn, diag0, tol, ndrop);
  }
  note_launch();
  k_negate<T><<<4 * num_sms(), 256, 0, s>>>(tiles, nti * CT * CT);
  SPNET_CUDA_TRY(cudaGetLastError());
  SPNET_CUDA_TRY(cudaMemcpyAsync(ndrop_out, ndrop, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  return SPNET_OK;
}

__global__ void k_round_tiles(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    b[q] = (float)a[q];
}

template <class T>
static int invert_impl(spnet_pc_s* pc, const double* A0) {
  cudaStream_t s = pc->op->stream;
  const int64_t m0 = pc->m0;
  const int nt = (int)((m0 + CT - 1) / CT);
  const int64_t nti = n_upper_tiles(nt);
  T* tiles = nullptr;
  SPNET_TRY(pc->mem.get(&tiles, nti * CT * CT));
  pc->ctiles = tiles;
  pc->ctiles_n = nt;
  int nd = 0;
  if constexpr (sizeof(T) == 8) {
    SPNET_TRY(sweep_inverse<T>(pc, A0, tiles, DROP64, &nd));
    pc->coarse_dropped = nd;
    return SPNET_OK;
  } else {
    SPNET_TRY(sweep_inverse<T>(pc, A0, tiles, TRIG32, &nd));
    pc->coarse_dropped = 0;
    if (nd == 0) return SPNET_OK;
    // a pivot at or below TRIG32: an ill-conditioned or singular A_0, inverted in FP64
    DevArena tmp;
    tmp.stream = s;
    struct Guard {
      DevArena& a;
      ~Guard() { a.free_all(); }
    } guard{tmp};
    double* t64 = nullptr;
    SPNET_TRY(tmp.get(&t64, nti * CT * CT));
    SPNET_TRY(sweep_inverse<double>(pc, A0, t64, DROP64, &nd));
    pc->coarse_dropped = nd;
    note_launch();
    k_round_tiles<<<4 * num_sms(), 256, 0, s>>>(t64, tiles, nti * CT * CT);
    SPNET_CUDA_TRY(cudaGetLastError());
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));
    return SPNET_OK;
  }
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
// Every part[R][K] has one writer; a second kernel sums part[R][0..nt-1] in K
// order into z_c (deterministic).
// ---------------------------------------------------------------------------
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
                                                     T* __restrict__ part, const int* done) {
  constexpr int RW = CT / 8;                  // rows per warp
  constexpr int RB = 8;                       // rows loaded per batch
  __shared__ T sI[CT], sJ[CT];
  __shared__ T scol[8][CT];
  pdl_wait();
  pdl_trigger();
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
}

// z_c[i] = sum over K of part[R][K][i - 128 R] in K order, R = i / 128
// (one thread per coarse dof; eight loads in flight)
template <class T>
__global__ void __launch_bounds__(256) k_coarse_reduce(int nt, int64_t m0, const T* __restrict__ part,
                                                       double* __restrict__ zc, const int* done) {
  pdl_wait();
  pdl_trigger();
  if (done && *done) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m0) return;
  const int64_t R = i / CT;
  const T* pr = part + R * nt * CT + (i - R * CT);
  double sum = 0.0;
  for (int K0 = 0; K0 < nt; K0 += 8) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = K0 + u < nt ? pr[(int64_t)(K0 + u) * CT] : T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (K0 + u < nt) sum += (double)v[u];
  }
  zc[i] = sum;
}

void launch_coarse_apply(spnet_pc_s* pc, const double* rc, double* zc, const int* done,
                         cudaStream_t s) {
  if (pc->m0 == 0) return;
  const unsigned tiles = (unsigned)n_upper_tiles(pc->ctiles_n);
  note_launch();
  note_launch();  // the product and its row reduction
  ProfScope ps(KID_COARSE, s);
  const unsigned rblocks = (unsigned)((pc->m0 + 255) / 256);
  if (pc->precision == SPNET_PREC_FP64) {
    launch_pdl(k_coarse_symv<double>, tiles, 256, 0, s, (const double*)pc->ctiles, pc->ctiles_n, (int64_t)pc->m0,
               rc, (const double*)pc->epart, (const int32_t*)pc->rtab, (double*)pc->cpart, done);
    launch_pdl(k_coarse_reduce<double>, rblocks, 256, 0, s, pc->ctiles_n, (int64_t)pc->m0,
               (const double*)pc->cpart, zc, done);
  } else {
    launch_pdl(k_coarse_symv<float>, tiles, 256, 0, s, (const float*)pc->ctiles, pc->ctiles_n, (int64_t)pc->m0,
               rc, (const double*)pc->epart, (const int32_t*)pc->rtab, (float*)pc->cpart, done);
    launch_pdl(k_coarse_reduce<float>, rblocks, 256, 0, s, pc->ctiles_n, (int64_t)pc->m0, (const float*)pc->cpart,
               zc, done);
  }
}

// ---------------------------------------------------------------------------
// The coarse solve for k right-hand sides at once (k <= 32): Z_c = A_0^{-1}
// R_0 R with blocks [coarse dof][k].  One block per stored tile stages the
// tile (rows padded), the restricted right-hand sides of its row block and of
// its column block in shared memory, and forms Z_IJ R_J (part [I][J]) and, off
// the diagonal, Z_IJ^T R_I (part [J][I]).  The restricted right-hand sides R_0 R
// are formed once per step by k_restrict_batch (each value summed over the corner
// sums of its mesh node in a fixed order) and read by the tiles as rows.  A thread owns UR rows (interleaved
// across the lanes: no bank conflicts on the padded tile) times JR
// right-hand sides and sums each over the tile's 128 columns in order, so a
// result does not depend on k.  A second kernel sums the parts of each row in
// tile order.  The tile is read once for all k.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t coarse_batch_smem(int vb, int kp) {
  return (size_t)vb * (CT * (CT + 1) + 2 * CT * kp);
}

template <int KP>
struct BatchTile {
  static constexpr int JR = KP < 4 ? KP : 4;                       // right-hand sides per thread
  static constexpr int UR = CT * KP / (256 * JR) > 1 ? CT * KP / (256 * JR) : 1;  // rows per thread
  static constexpr int TPG = CT / UR;                              // threads per group of JR columns
  static constexpr int ACTIVE = TPG * (KP / JR);                   // threads with work (<= 256)
};

// RC[ci][j] = (R_0 R)[ci][j] from the element corner sums EP [entries][k]
template <class T>
__global__ void __launch_bounds__(256) k_restrict_batch(int64_t m0, int k, const double* __restrict__ EP,
                                                        const int32_t* __restrict__ rtab, T* __restrict__ RC,
                                                        const int* done) {
  pdl_wait();
  pdl_trigger();
  if (done && *done) return;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m0 * k) return;
  const int64_t ci = q / k;
  const int j = (int)(q % k);
  double sum = 0.0;
#pragma unroll
  for (int cp = 0; cp < 8; ++cp) {
    const int off = rtab[8 * ci + cp];
    if (off >= 0) sum += EP[(int64_t)off * k + j];
  }
  RC[q] = (T)sum;
}

template <class T, int KP>
__global__ void __launch_bounds__(256) k_coarse_batch(const T* __restrict__ tiles, int nt, int64_t m0, int k,
                                                      const T* __restrict__ RC, T* __restrict__ part,
                                                      const int* done) {
  using BT = BatchTile<KP>;
  extern __shared__ __align__(16) char sm_cb[];
  T (*Zs)[CT + 1] = reinterpret_cast<T (*)[CT + 1]>(sm_cb);
  T* sI = reinterpret_cast<T*>(sm_cb + sizeof(T) * CT * (CT + 1));
  T* sJ = sI + CT * KP;
  pdl_wait();
  pdl_trigger();
  if (done && *done) return;
  int I, J;
  upper_tile(blockIdx.x, nt, &I, &J);
  const T* Zt = tiles + (int64_t)blockIdx.x * CT * CT;
  for (int q = threadIdx.x; q < CT * CT; q += blockDim.x) Zs[q / CT][q % CT] = Zt[q];
  // the restricted right-hand sides of the tile's row and column blocks
  for (int q = threadIdx.x; q < 2 * CT * KP; q += blockDim.x) {
    const int side = q / (CT * KP), u = (q / KP) % CT, j = q % KP;
    const int64_t ci = (int64_t)(side == 0 ? I : J) * CT + u;
    (side == 0 ? sI : sJ)[u * KP + j] = (ci < m0 && j < k) ? RC[ci * k + j] : T(0);
  }
  __syncthreads();
  if ((int)threadIdx.x >= BT::ACTIVE) return;  // no barrier follows
  const int g = threadIdx.x / BT::TPG, ut = threadIdx.x % BT::TPG;
  const int j0 = g * BT::JR;
  {  // part[I][J][u][j] = sum_c Z[u][c] R_J[c][j]
    T acc[BT::UR][BT::JR];
#pragma unroll
    for (int a = 0; a < BT::UR; ++a)
#pragma unroll
      for (int b = 0; b < BT::JR; ++b) acc[a][b] = T(0);
    for (int c = 0; c < CT; ++c) {
      T rv[BT::JR];
#pragma unroll
      for (int b = 0; b < BT::JR; ++b) rv[b] = sJ[c * KP + j0 + b];
#pragma unroll
      for (int a = 0; a < BT::UR; ++a) {
        const T z = Zs[ut + a * BT::TPG][c];
#pragma unroll
        for (int b = 0; b < BT::JR; ++b) acc[a][b] = fma(z, rv[b], acc[a][b]);
      }
    }
    T* out = part + ((int64_t)I * nt + J) * CT * KP;
#pragma unroll
    for (int a = 0; a < BT::UR; ++a)
#pragma unroll
      for (int b = 0; b < BT::JR; ++b) out[(ut + a * BT::TPG) * KP + j0 + b] = acc[a][b];
  }
  if (I != J) {  // part[J][I][c][j] = sum_u Z[u][c] R_I[u][j]
    T acc[BT::UR][BT::JR];
#pragma unroll
    for (int a = 0; a < BT::UR; ++a)
#pragma unroll
      for (int b = 0; b < BT::JR; ++b) acc[a][b] = T(0);
    for (int u = 0; u < CT; ++u) {
      T rv[BT::JR];
#pragma unroll
      for (int b = 0; b < BT::JR; ++b) rv[b] = sI[u * KP + j0 + b];
#pragma unroll
      for (int a = 0; a < BT::UR; ++a) {
        const T z = Zs[u][ut + a * BT::TPG];
#pragma unroll
        for (int b = 0; b < BT::JR; ++b) acc[a][b] = fma(z, rv[b], acc[a][b]);
      }
    }
    T* out = part + ((int64_t)J * nt + I) * CT * KP;
#pragma unroll
    for (int a = 0; a < BT::UR; ++a)
#pragma unroll
      for (int b = 0; b < BT::JR; ++b) out[(ut + a * BT::TPG) * KP + j0 + b] = acc[a][b];
  }
}

// zc[i][j] = sum over K of part[R][K][i - 128 R][j] in K order, R = i / 128
template <class T>
__global__ void __launch_bounds__(256) k_coarse_batch_reduce(int nt, int64_t m0, int k, int kp,
                                                             const T* __restrict__ part, double* __restrict__ zc,
                                                             const int* done) {
  pdl_wait();
  pdl_trigger();
  if (done && *done) return;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m0 * k) return;
  const int64_t i = q / k;
  const int j = (int)(q % k);
  const int64_t R = i / CT;
  const T* pr = part + (R * nt * CT + (i - R * CT)) * kp + j;
  double sum = 0.0;
  for (int K0 = 0; K0 < nt; K0 += 8) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = K0 + u < nt ? pr[(int64_t)(K0 + u) * CT * kp] : T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (K0 + u < nt) sum += (double)v[u];
  }
  zc[q] = sum;
}

// bytes of the parts of the k-right-hand-side coarse product, then the restricted block RC [m0][k]
static size_t parts_only_bytes(const spnet_pc_s* pc, int kp, int vb) {
  return ((size_t)vb * pc->ctiles_n * pc->ctiles_n * CT * kp + 255) / 256 * 256;
}
size_t coarse_batch_part_bytes(const spnet_pc_s* pc, int k) {
  const int kp = k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
  const int vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  return parts_only_bytes(pc, kp, vb) + (size_t)vb * pc->m0 * k;
}

template <class T, int KP>
static int coarse_batch_t(spnet_pc_s* pc, const double* EP, int k, double* ZC, void* part, const int* done,
                          cudaStream_t s) {
  static std::atomic<bool> attr_set[64];  // per device
  int dev = 0;
  SPNET_CUDA_TRY(cudaGetDevice(&dev));
  dev &= 63;
  const size_t smem = coarse_batch_smem((int)sizeof(T), KP);
  if (!attr_set[dev]) {
    SPNET_CUDA_TRY(cudaFuncSetAttribute(k_coarse_batch<T, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set[dev] = true;
  }
  const unsigned tiles = (unsigned)n_upper_tiles(pc->ctiles_n);
  const unsigned rblocks = (unsigned)((pc->m0 * k + 255) / 256);
  T* RC = (T*)((char*)part + parts_only_bytes(pc, KP, (int)sizeof(T)));
  launch_pdl(k_restrict_batch<T>, rblocks, 256, 0, s, (int64_t)pc->m0, k, EP, (const int32_t*)pc->rtab, RC, done);
  launch_pdl(k_coarse_batch<T, KP>, tiles, 256, smem, s, (const T*)pc->ctiles, pc->ctiles_n, (int64_t)pc->m0, k,
             (const T*)RC, (T*)part, done);
  launch_pdl(k_coarse_batch_reduce<T>, rblocks, 256, 0, s, pc->ctiles_n, (int64_t)pc->m0, k, KP, (const T*)part, ZC,
             done);
  return SPNET_OK;
}

template <class T>
static int coarse_batch_p(spnet_pc_s* pc, const double* EP, int k, double* ZC, void* part, const int* done,
                          cudaStream_t s) {
  if (k <= 1) return coarse_batch_t<T, 1>(pc, EP, k, ZC, part, done, s);
  if (k <= 2) return coarse_batch_t<T, 2>(pc, EP, k, ZC, part, done, s);
  if (k <= 4) return coarse_batch_t<T, 4>(pc, EP, k, ZC, part, done, s);
  if (k <= 8) return coarse_batch_t<T, 8>(pc, EP, k, ZC, part, done, s);
  if (k <= 16) return coarse_batch_t<T, 16>(pc, EP, k, ZC, part, done, s);
  return coarse_batch_t<T, 32>(pc, EP, k, ZC, part, done, s);
}

// ZC [m0][k] = A_0^{-1} R_0 R from the element corner sums EP [corner entries][k]
int launch_coarse_batch(spnet_pc_s* pc, const double* EP, int k, double* ZC, void* part, const int* done,
                        cudaStream_t s) {
  if (pc->m0 == 0) return SPNET_OK;
  if (k < 1 || k > 32) return fail(SPNET_ERR_BAD_INPUT, "coarse solve: 1..32 right-hand sides at once");
  note_launch();
  note_launch();
  note_launch();  // the restriction, the product and its row reduction
  ProfScope ps(KID_COARSE, s);
  if (pc->precision == SPNET_PREC_FP64) return coarse_batch_p<double>(pc, EP, k, ZC, part, done, s);
  return coarse_batch_p<float>(pc, EP, k, ZC, part, done, s);
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

// the partial products, their counters and the restriction table of the product
template <class T>
static int prepare_product(spnet_pc_s* pc) {
  cudaStream_t s = pc->op->stream;
  const int nt = pc->ctiles_n;
  T* part = nullptr;
  SPNET_TRY(pc->mem.get(&part, (int64_t)nt * nt * CT));
  const int64_t nmc = (int64_t)pc->n_mesh * pc->ndof;
  if ((int64_t)pc->n_elem * pc->nc * pc->ndof > INT32_MAX)
    return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: too many element corner sums for 32-bit offsets");
  SPNET_TRY(pc->mem.get(&pc->rtab, 8ll * pc->m0));
  note_launch();
  k_restrict_table<<<(unsigned)((nmc + 255) / 256), 256, 0, s>>>(nmc, mesh_of_pc(pc), pc->ndof, pc->cidx, pc->rtab);
  SPNET_CUDA_TRY(cudaGetLastError());
  pc->cpart = part;
  return SPNET_OK;
}

int coarse_gemv_prepare(spnet_pc_s* pc) {
  if (pc->m0 == 0) return SPNET_OK;
  if (pc->precision == SPNET_PREC_FP64) return prepare_product<double>(pc);
  return prepare_product<float>(pc);
}

}  // namespace spnet
