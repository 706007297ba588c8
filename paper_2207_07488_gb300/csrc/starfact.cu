// Exact local solves on the stars (Section 4.1, eq. defPj):
//   A_j = E_j^T A E_j,   w_j = A_j^{-1} E_j^T r,
// for every star j at once, one warp per star.
//
// Each A_j is factored A_j = L_j L_j^T (sparse Cholesky) in an elimination
// order built in rounds: every round eliminates an independent set of nodes of
// small degree in the current elimination graph (their fill is added before
// the next round).  Nodes eliminated in one round do not couple in L, so a
// round is a level of the triangular solves: all rows of a level are solved
// in parallel by the lanes of the warp, and a star of a few hundred dofs needs
// a few dozen dependent steps instead of one per row.  When the remaining
// graph gets dense (a degree above SWITCH_DEG, or an adjacency list full),
// the rest is eliminated as a dense block, one node per level.
//
// Pass 1 (symbolic) computes the order, levels and the structure of L in
// column form (for the backward solve) and in row form (forward solve) and
// places each star's blob in a pool; pass 2 (numeric) fills the values level
// by level, every lane computing one column left-looking in FP64.  Values are
// kept in FP64 and rounded to FP32 for the mixed-precision solve.
#include <cmath>

#include "spnet_internal.cuh"

namespace spnet {

constexpr int CAP = 32;          // adjacency slots per node during elimination
constexpr int SWITCH_DEG = 24;   // minimum degree above which the rest is dense
constexpr int CORE_MAX = 256;    // largest dense block handled
constexpr int CORE_ENTRIES = CORE_MAX * (CORE_MAX - 1) / 2;

// A star's blob: a compact "solve section" (all the triangular solves read)
// followed by a set-up section.  Values of the solve section are FP64 or FP32
// (vbytes); the set-up section holds the column->row entry map and, for FP32
// solves, the FP64 factor computed first.
struct BlobLayout {
  int64_t gidx, rowptr, colptr, lvl, perm, rowidx, colidx, rowval, colval, invd, solve;
  int64_t c2r, v64, total;
};

__host__ __device__ inline int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline BlobLayout blob_layout(int n, int nlev, int nnz, int vbytes) {
  BlobLayout L;
  int64_t o = 16;  // header: n, nlev, nnz, 0
  L.gidx = o;   o += 4ll * n;
  L.rowptr = o; o += 4ll * (n + 1);
  L.colptr = o; o += 4ll * (n + 1);
  L.lvl = o;    o += 2ll * (nlev + 1);
  L.perm = o;   o += 2ll * n;
  L.rowidx = o; o += 2ll * nnz;
  L.colidx = o; o += 2ll * nnz;
  o = align_up(o, 8);
  L.rowval = o; o += (int64_t)vbytes * nnz;
  L.colval = o; o += (int64_t)vbytes * nnz;
  L.invd = o;   o += (int64_t)vbytes * n;
  L.solve = align_up(o, 16);
  o = L.solve;
  L.c2r = o;    o += 4ll * nnz;
  o = align_up(o, 8);
  L.v64 = vbytes == 8 ? L.rowval : o;       // FP64 row values, col values, 1/L_vv
  if (vbytes != 8) o += 8ll * (2ll * nnz + n);
  L.total = align_up(o, 16);
  return L;
}

struct StarArgs {
  Mesh m;
  int S;
  const int32_t* star_mesh;
  const int32_t* star_n;
  const int32_t* elem_ptr;
  const int32_t* elem_of;
  const int64_t* kptr;
  const int32_t* kcol;
  const double* kval;
  char* scratch;
  int64_t stride;  // global scratch bytes per warp
  int64_t hot;     // hot bytes per warp
  int hot_in_smem; // 1: hot arrays in dynamic shared memory
  int nmax;
  char* pool;
  int64_t pool_cap;
  unsigned long long* pool_top;
  int64_t* star_off;
  int32_t* star_lev;
  int32_t* star_nnz;
  int* flags;
  int* next;
  int vbytes;
};

struct Scratch {
  uint16_t* nbr;     // [nmax*CAP]
  uint16_t* colent;  // [nmax*CAP + CORE_ENTRIES]
  int32_t* deg;      // [nmax]
  int32_t* state;    // [nmax]: -1 alive, else elimination position
  int32_t* posnode;  // [nmax]
  int32_t* colstart; // [nmax+1]
  int32_t* lvl;      // [nmax+1]
  int32_t* rcnt;     // [nmax+1]
  int32_t* rstart;   // [nmax+1]
  uint8_t* sel;      // [nmax]
};

// hot arrays (adjacency, degrees, states, selection), touched in every round:
// in shared memory when they fit, else with the cold ones in global scratch
__host__ __device__ inline int64_t hot_bytes(int nmax) {
  return align_up(2ll * nmax * CAP, 16) + align_up(8ll * nmax, 16) + align_up((int64_t)nmax, 16);
}

__host__ __device__ inline int64_t cold_bytes(int nmax) {
  int64_t o = 2ll * ((int64_t)nmax * CAP + CORE_ENTRIES);
  o = align_up(o, 8);
  o += 4ll * (nmax + 1) * 6;
  return align_up(o, 256);
}

__device__ inline Scratch carve(char* cold, char* hot, int nmax) {
  Scratch s;
  int64_t o = 0;
  s.nbr = (uint16_t*)(hot + o);   o = align_up(o + 2ll * nmax * CAP, 16);
  s.deg = (int32_t*)(hot + o);    o += 4ll * nmax;
  s.state = (int32_t*)(hot + o);  o = align_up(o + 4ll * nmax, 16);
  s.sel = (uint8_t*)(hot + o);
  o = 0;
  s.colent = (uint16_t*)(cold + o); o += 2ll * ((int64_t)nmax * CAP + CORE_ENTRIES);
  o = align_up(o, 8);
  s.posnode = (int32_t*)(cold + o);  o += 4ll * (nmax + 1);
  s.colstart = (int32_t*)(cold + o); o += 4ll * (nmax + 1);
  s.lvl = (int32_t*)(cold + o);      o += 4ll * (nmax + 1);
  s.rcnt = (int32_t*)(cold + o);     o += 4ll * (nmax + 1);
  s.rstart = (int32_t*)(cold + o);   o += 4ll * (nmax + 1);
  return s;
}

// the 2^d elements of a star, in c' order, with their offsets in the star
struct StarElems {
  int e[8];
  int off[9];
  int nc;
};

__device__ inline StarElems star_elems(const Mesh& m, int k, const int32_t* elem_ptr) {
  StarElems se;
  int km[3];
  mesh_multi(m, k, km);
  int o = 0;
  se.nc = m.nc;
  for (int cp = 0; cp < m.nc; ++cp) {
    int e = elem_around(m, km, cp);
    se.e[cp] = e;
    se.off[cp] = o;
    if (e >= 0) o += elem_ptr[e + 1] - elem_ptr[e];
  }
  se.off[m.nc] = o;
  return se;
}

__device__ inline int pc_of_local(const StarElems& se, const int32_t* elem_ptr, int t) {
  int cp = 0;
  while (cp + 1 < se.nc && se.off[cp + 1] <= t) ++cp;
  return elem_ptr[se.e[cp]] + (t - se.off[cp]);
}

__device__ inline int local_of_pc(const Mesh& m, const StarElems& se, const int32_t* elem_ptr,
                                  const int32_t* elem_of, int k_multi0, int k_multi1, int k_multi2,
                                  int j) {
  int e = elem_of[j];
  int ex[3];
  elem_multi(m, e, ex);
  int km[3] = {k_multi0, k_multi1, k_multi2};
  int cp = 0;
  for (int a = 0; a < m.d; ++a) {
    int r = ex[a] - (km[a] - 1);
    if (r < 0 || r > 1) return -1;
    cp |= r << a;
  }
  return se.off[cp] + (j - elem_ptr[e]);
}

__device__ inline int warp_min(int v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ inline int warp_sum(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline int warp_incl_scan(int v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// remove eliminated neighbours from the adjacency list of every alive node
__device__ inline void compact_all(const Scratch& W, int n, int lane) {
  for (int t = lane; t < n; t += 32) {
    if (W.state[t] >= 0) continue;
    uint16_t* lst = W.nbr + (int64_t)t * CAP;
    int c = 0, d = W.deg[t];
    for (int q = 0; q < d; ++q) {
      int u = lst[q];
      if (W.state[u] < 0) lst[c++] = (uint16_t)u;
    }
    W.deg[t] = c;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(128) k_star_symbolic(StarArgs A) {
  extern __shared__ __align__(16) char sm_hot[];
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  char* cold = A.scratch + wg * A.stride;
  char* hot = A.hot_in_smem ? sm_hot + (threadIdx.x >> 5) * A.hot : cold + cold_bytes(A.nmax);
  const Scratch W = carve(cold, hot, A.nmax);
  const unsigned FULL = 0xffffffffu;
  for (;;) {
    int s = 0;
    if (lane == 0) s = atomicAdd(A.next, 1);
    s = __shfl_sync(FULL, s, 0);
    if (s >= A.S) break;
    const int k = A.star_mesh[s];
    const int n = A.star_n[s];
    if (n > A.nmax || n > 65535) {
      if (lane == 0) atomicOr(A.flags, FLAG_STAR_BIG);
      continue;
    }
    const StarElems se = star_elems(A.m, k, A.elem_ptr);
    int km[3];
    mesh_multi(A.m, k, km);
    // adjacency of the star graph
    bool ovf = false;
    for (int t = lane; t < n; t += 32) {
      int i = pc_of_local(se, A.elem_ptr, t);
      int cnt = 0;
      for (int64_t q = A.kptr[i]; q < A.kptr[i + 1]; ++q) {
        int j = A.kcol[q];
        if (j == i) continue;
        int lt = local_of_pc(A.m, se, A.elem_ptr, A.elem_of, km[0], km[1], km[2], j);
        if (lt < 0) continue;
        if (cnt < CAP) W.nbr[(int64_t)t * CAP + cnt++] = (uint16_t)lt;
        else ovf = true;
      }
      W.deg[t] = cnt;
      W.state[t] = -1;
    }
    ovf = __any_sync(FULL, ovf);
    __syncwarp();
    int npos = 0, nlev = 0, ncol = 0;
    bool dense = ovf;
    while (!dense && npos < n) {
      compact_all(W, n, lane);
      int md = 1 << 30;
      for (int t = lane; t < n; t += 32)
        if (W.state[t] < 0) md = min(md, W.deg[t]);
      md = warp_min(md);
      if (md > SWITCH_DEG) {
        dense = true;
        break;
      }
      const int thr = max(md, 2);
      // independent set: candidates of degree <= thr that beat every candidate neighbour
      for (int t = lane; t < n; t += 32) {
        bool sl = false;
        if (W.state[t] < 0 && W.deg[t] <= thr) {
          sl = true;
          const int dt = W.deg[t];
          const uint16_t* lst = W.nbr + (int64_t)t * CAP;
          for (int q = 0; q < dt; ++q) {
            int u = lst[q];
            int du = W.deg[u];
            if (du <= thr && (du < dt || (du == dt && u < t))) {
              sl = false;
              break;
            }
          }
        }
        W.sel[t] = sl ? 1 : 0;
      }
      __syncwarp();
      // positions in ascending node order, columns = current neighbour lists
      const int lev_start = npos;
      W.lvl[nlev] = npos;
      for (int base = 0; base < n; base += 32) {
        int t = base + lane;
        bool sl = t < n && W.sel[t];
        unsigned b = __ballot_sync(FULL, sl);
        int dcount = sl ? W.deg[t] : 0;
        int incl = warp_incl_scan(dcount, lane);
        int tot = __shfl_sync(FULL, incl, 31);
        if (sl) {
          int pos = npos + __popc(b & ((1u << lane) - 1u));
          int cs = ncol + incl - dcount;
          W.posnode[pos] = t;
          W.colstart[pos] = cs;
          const uint16_t* lst = W.nbr + (int64_t)t * CAP;
          for (int q = 0; q < dcount; ++q) W.colent[cs + q] = lst[q];
          W.state[t] = pos;
        }
        npos += __popc(b);
        ncol += tot;
      }
      W.colstart[npos] = ncol;
      __syncwarp();
      compact_all(W, n, lane);
      // fill among the neighbours of each eliminated node (serial, lane-parallel lookups)
      bool full = false;
      for (int pos = lev_start; pos < npos; ++pos) {
        const int cs = W.colstart[pos], ce = W.colstart[pos + 1];
        for (int ai = cs; ai < ce; ++ai) {
          for (int bi = ai + 1; bi < ce; ++bi) {
            const int a = W.colent[ai], b = W.colent[bi];
            const int da = W.deg[a];
            bool found = false;
            for (int q = lane; q < da; q += 32) found |= (W.nbr[(int64_t)a * CAP + q] == b);
            found = __any_sync(FULL, found);
            if (!found) {
              if (lane == 0) {
                int db = W.deg[b];
                if (da < CAP && db < CAP) {
                  W.nbr[(int64_t)a * CAP + da] = (uint16_t)b;
                  W.deg[a] = da + 1;
                  W.nbr[(int64_t)b * CAP + db] = (uint16_t)a;
                  W.deg[b] = db + 1;
                } else {
                  full = true;
                }
              }
              __syncwarp();
            }
          }
        }
      }
      full = __shfl_sync(FULL, (int)full, 0) != 0;
      nlev++;
      if (full) dense = true;
    }
    if (dense && npos < n) {
      // the rest, in ascending node order, one node per level, columns dense
      const int core0 = npos;
      for (int base = 0; base < n; base += 32) {
        int t = base + lane;
        bool al = t < n && W.state[t] < 0;
        unsigned b = __ballot_sync(FULL, al);
        if (al) {
          int pos = npos + __popc(b & ((1u << lane) - 1u));
          W.posnode[pos] = t;
          W.state[t] = pos;
        }
        npos += __popc(b);
      }
      const int c = n - core0;
      if (c > CORE_MAX || ncol + c * (c - 1) / 2 > A.nmax * CAP + CORE_ENTRIES) {
        if (lane == 0) atomicOr(A.flags, FLAG_STAR_BIG);
        continue;
      }
      for (int q = 0; q < c; ++q) {
        W.lvl[nlev + q] = core0 + q;
        int cs = ncol + q * (c - 1) - q * (q - 1) / 2;
        if (lane == 0) W.colstart[core0 + q] = cs;
        for (int r = q + 1 + lane; r < c; r += 32) W.colent[cs + (r - q - 1)] = (uint16_t)W.posnode[core0 + r];
      }
      nlev += c;
      ncol += c * (c - 1) / 2;
      if (lane == 0) W.colstart[n] = ncol;
      __syncwarp();
    }
    if (lane == 0) W.lvl[nlev] = n;
    // column entries to positions; row counts
    for (int t = lane; t <= n; t += 32) W.rcnt[t] = 0;
    __syncwarp();
    for (int q = lane; q < ncol; q += 32) {
      int pos = W.state[W.colent[q]];
      W.colent[q] = (uint16_t)pos;
      atomicAdd(&W.rcnt[pos], 1);
    }
    __syncwarp();
    int carry = 0;
    for (int base = 0; base < n; base += 32) {
      int t = base + lane;
      int v = t < n ? W.rcnt[t] : 0;
      int incl = warp_incl_scan(v, lane);
      if (t < n) W.rstart[t] = carry + incl - v;
      carry += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) W.rstart[n] = carry;
    for (int t = lane; t < n; t += 32) W.rcnt[t] = 0;
    __syncwarp();
    // place the blob
    const BlobLayout L = blob_layout(n, nlev, ncol, A.vbytes);
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(A.pool_top, (unsigned long long)L.total);
    off = __shfl_sync(FULL, off, 0);
    if ((int64_t)off + L.total > A.pool_cap) {
      if (lane == 0) atomicOr(A.flags, FLAG_POOL);
      continue;
    }
    char* blob = A.pool + off;
    if (lane == 0) {
      int32_t* hdr = (int32_t*)blob;
      hdr[0] = n;
      hdr[1] = nlev;
      hdr[2] = ncol;
      hdr[3] = 0;
      A.star_off[s] = (int64_t)off;
      A.star_lev[s] = nlev;
      A.star_nnz[s] = ncol;
    }
    int32_t* gidx = (int32_t*)(blob + L.gidx);
    uint16_t* perm = (uint16_t*)(blob + L.perm);
    uint16_t* lvl = (uint16_t*)(blob + L.lvl);
    uint32_t* colptr = (uint32_t*)(blob + L.colptr);
    uint16_t* colidx = (uint16_t*)(blob + L.colidx);
    uint32_t* rowptr = (uint32_t*)(blob + L.rowptr);
    uint16_t* rowidx = (uint16_t*)(blob + L.rowidx);
    int32_t* c2r = (int32_t*)(blob + L.c2r);
    for (int pos = lane; pos < n; pos += 32) {
      int t = W.posnode[pos];
      gidx[pos] = pc_of_local(se, A.elem_ptr, t);
      perm[pos] = (uint16_t)t;
    }
    for (int q = lane; q <= nlev; q += 32) lvl[q] = (uint16_t)W.lvl[q];
    for (int q = lane; q <= n; q += 32) {
      colptr[q] = (uint32_t)W.colstart[q];
      rowptr[q] = (uint32_t)W.rstart[q];
    }
    for (int q = lane; q < ncol; q += 32) colidx[q] = W.colent[q];
    // row form: columns in ascending position, so every row lists its columns ascending
    for (int v = 0; v < n; ++v) {
      const int cs = W.colstart[v], ce = W.colstart[v + 1];
      for (int q = cs + lane; q < ce; q += 32) {
        int i = W.colent[q];
        int slot = W.rstart[i] + W.rcnt[i];
        W.rcnt[i] += 1;
        rowidx[slot] = (uint16_t)v;
        c2r[q] = slot;
      }
      __syncwarp();
    }
    __syncwarp();
  }
}

__device__ inline double k_entry(const int64_t* kptr, const int32_t* kcol, const double* kval, int row,
                                 int col) {
  int64_t lo = kptr[row], hi = kptr[row + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) >> 1;
    int c = kcol[mid];
    if (c == col) return kval[mid];
    if (c < col) lo = mid + 1; else hi = mid - 1;
  }
  return 0.0;
}

__global__ void __launch_bounds__(128) k_star_numeric(int S, char* pool, const int64_t* star_off,
                                                      const int64_t* kptr, const int32_t* kcol,
                                                      const double* kval, int vbytes, int* flags) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nw) {
    char* blob = pool + star_off[s];
    const int32_t* hdr = (const int32_t*)blob;
    const int n = hdr[0], nlev = hdr[1], nnz = hdr[2];
    const BlobLayout L = blob_layout(n, nlev, nnz, vbytes);
    const int32_t* gidx = (const int32_t*)(blob + L.gidx);
    const uint16_t* lvl = (const uint16_t*)(blob + L.lvl);
    const uint32_t* colptr = (const uint32_t*)(blob + L.colptr);
    const uint16_t* colidx = (const uint16_t*)(blob + L.colidx);
    const uint32_t* rowptr = (const uint32_t*)(blob + L.rowptr);
    const uint16_t* rowidx = (const uint16_t*)(blob + L.rowidx);
    const int32_t* c2r = (const int32_t*)(blob + L.c2r);
    double* rowv = (double*)(blob + L.v64);
    double* colv = rowv + nnz;
    double* invd = colv + nnz;
    bool bad = false;
    for (int l = 0; l < nlev; ++l) {
      for (int v = lvl[l] + lane; v < (int)lvl[l + 1]; v += 32) {
        const int gv = gidx[v];
        double d = k_entry(kptr, kcol, kval, gv, gv);
        for (uint32_t q = rowptr[v]; q < rowptr[v + 1]; ++q) d -= rowv[q] * rowv[q];
        if (!(d > 0.0)) {
          bad = true;
          d = 1.0;
        }
        const double inv = 1.0 / sqrt(d);
        invd[v] = inv;
        const uint32_t rv0 = rowptr[v], rv1 = rowptr[v + 1];
        for (uint32_t q = colptr[v]; q < colptr[v + 1]; ++q) {
          const int i = colidx[q];
          double a = k_entry(kptr, kcol, kval, gv, gidx[i]);
          uint32_t kv = rv0, ki = rowptr[i];
          const uint32_t ki1 = rowptr[i + 1];
          while (kv < rv1 && ki < ki1) {
            const int uv = rowidx[kv], ui = rowidx[ki];
            if (uv == ui) {
              a -= rowv[kv] * rowv[ki];
              ++kv;
              ++ki;
            } else if (uv < ui) {
              ++kv;
            } else {
              ++ki;
            }
          }
          const double lval = a * inv;
          colv[q] = lval;
          rowv[c2r[q]] = lval;
        }
      }
      __syncwarp();
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_NOT_SPD);
    if (vbytes == 4) {
      float* r32 = (float*)(blob + L.rowval);
      for (int q = lane; q < 2 * nnz + n; q += 32) r32[q] = (float)rowv[q];
    }
  }
}

// ---------------------------------------------------------------------------
// The solve works on compact per-star sections packed in star order:
//   header (80 B): n, nlev, nnz, pointer bytes; base of the star in w; the pc
//                  index of the first dof and the local offset of each of the
//                  star's 2^d elements
//   lvl [nlev+1] u16, perm [n] u16, rowptr/colptr [n+1] (u16, or u32 when
//   nnz > 65535), rowidx/colidx [nnz] u16, then (8-byte aligned) row values,
//   column values and 1/L_vv in the solve precision; padded to 16 bytes.
// Stars are grouped into blocks whose sections and vectors fit a shared-memory
// budget; a block copies its contiguous sections into shared memory with
// 16-byte loads and each warp then solves one star there: every level step
// reads shared memory only.
// ---------------------------------------------------------------------------
constexpr int SOLVE_WPB = 12;                  // warps (stars) per block
constexpr int SOLVE_BUDGET = 110 * 1024;       // shared memory per block
constexpr int SEC_HDR = 80;

struct SecLayout {
  int64_t lvl, perm, rowptr, colptr, rowidx, colidx, rowval, colval, invd, total;
};

__host__ __device__ inline SecLayout sec_layout(int n, int nlev, int nnz, int vb) {
  SecLayout L;
  const int pw = nnz > 65535 ? 4 : 2;
  int64_t o = SEC_HDR;
  L.lvl = o;    o += 2ll * (nlev + 1);
  L.perm = o;   o += 2ll * n;
  o = align_up(o, pw);
  L.rowptr = o; o += (int64_t)pw * (n + 1);
  L.colptr = o; o += (int64_t)pw * (n + 1);
  L.rowidx = o; o += 2ll * nnz;
  L.colidx = o; o += 2ll * nnz;
  o = align_up(o, 8);
  L.rowval = o; o += (int64_t)vb * nnz;
  L.colval = o; o += (int64_t)vb * nnz;
  L.invd = o;   o += (int64_t)vb * n;
  L.total = align_up(o, 16);
  return L;
}

__global__ void k_sec_sizes(int S, const char* pool, const int64_t* star_off, int vb, int64_t* sz,
                            int32_t* yb) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const int32_t* h = (const int32_t*)(pool + star_off[s]);
    sz[s] = sec_layout(h[0], h[1], h[2], vb).total;
    yb[s] = (int32_t)align_up((int64_t)vb * h[0], 16);
  }
}

// warp per star: setup blob (FP64) -> compact section (vb-byte values)
template <class T>
__global__ void k_sec_pack(int S, Mesh m, const char* pool, const int64_t* star_off,
                           const int32_t* star_mesh, const int32_t* elem_ptr, const int64_t* star_ptr,
                           char* spool, const int64_t* soff) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nw) {
    const char* blob = pool + star_off[s];
    const int32_t* hb = (const int32_t*)blob;
    const int n = hb[0], nlev = hb[1], nnz = hb[2];
    const BlobLayout B = blob_layout(n, nlev, nnz, 8);
    const SecLayout L = sec_layout(n, nlev, nnz, sizeof(T));
    char* sec = spool + soff[s];
    if (lane == 0) {
      int32_t* h = (int32_t*)sec;
      h[0] = n;
      h[1] = nlev;
      h[2] = nnz;
      h[3] = nnz > 65535 ? 4 : 2;
      *(int64_t*)(sec + 16) = star_ptr[s];
      int32_t* es = (int32_t*)(sec + 24);
      uint16_t* eo = (uint16_t*)(sec + 56);
      const StarElems se = star_elems(m, star_mesh[s], elem_ptr);
      for (int cp = 0; cp < 8; ++cp) es[cp] = (cp < m.nc && se.e[cp] >= 0) ? elem_ptr[se.e[cp]] : -1;
      for (int cp = 0; cp <= 8; ++cp) eo[cp] = (uint16_t)(cp <= m.nc ? se.off[cp < m.nc ? cp : m.nc] : n);
    }
    const uint16_t* lvl = (const uint16_t*)(blob + B.lvl);
    const uint16_t* perm = (const uint16_t*)(blob + B.perm);
    const uint32_t* rowptr = (const uint32_t*)(blob + B.rowptr);
    const uint32_t* colptr = (const uint32_t*)(blob + B.colptr);
    const uint16_t* rowidx = (const uint16_t*)(blob + B.rowidx);
    const uint16_t* colidx = (const uint16_t*)(blob + B.colidx);
    const double* v64 = (const double*)(blob + B.v64);  // row values, column values, 1/L_vv
    for (int q = lane; q <= nlev; q += 32) ((uint16_t*)(sec + L.lvl))[q] = lvl[q];
    for (int q = lane; q < n; q += 32) ((uint16_t*)(sec + L.perm))[q] = perm[q];
    if (nnz > 65535) {
      for (int q = lane; q <= n; q += 32) {
        ((uint32_t*)(sec + L.rowptr))[q] = rowptr[q];
        ((uint32_t*)(sec + L.colptr))[q] = colptr[q];
      }
    } else {
      for (int q = lane; q <= n; q += 32) {
        ((uint16_t*)(sec + L.rowptr))[q] = (uint16_t)rowptr[q];
        ((uint16_t*)(sec + L.colptr))[q] = (uint16_t)colptr[q];
      }
    }
    for (int q = lane; q < nnz; q += 32) {
      ((uint16_t*)(sec + L.rowidx))[q] = rowidx[q];
      ((uint16_t*)(sec + L.colidx))[q] = colidx[q];
    }
    T* vals = (T*)(sec + L.rowval);  // rowval, colval, invd are contiguous
    for (int q = lane; q < 2 * nnz + n; q += 32) vals[q] = (T)v64[q];
  }
}

template <class T, class PT>
__device__ __forceinline__ void solve_section(const char* sec, T* y, const double* __restrict__ r,
                                              double* __restrict__ w, int lane) {
  const int32_t* h = (const int32_t*)sec;
  const int n = h[0], nlev = h[1], nnz = h[2];
  const SecLayout L = sec_layout(n, nlev, nnz, sizeof(T));
  const int64_t base = *(const int64_t*)(sec + 16);
  const int32_t* es = (const int32_t*)(sec + 24);
  const uint16_t* eo = (const uint16_t*)(sec + 56);
  const uint16_t* lvl = (const uint16_t*)(sec + L.lvl);
  const uint16_t* perm = (const uint16_t*)(sec + L.perm);
  const PT* rowptr = (const PT*)(sec + L.rowptr);
  const PT* colptr = (const PT*)(sec + L.colptr);
  const uint16_t* rowidx = (const uint16_t*)(sec + L.rowidx);
  const uint16_t* colidx = (const uint16_t*)(sec + L.colidx);
  const T* rowv = (const T*)(sec + L.rowval);
  const T* colv = (const T*)(sec + L.colval);
  const T* invd = (const T*)(sec + L.invd);
  // gather r over the star: position -> element-concatenated index -> pc index
  constexpr int GU = 4;
  for (int p0 = 0; p0 < n; p0 += 32 * GU) {
    double rv[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int pos = p0 + u * 32 + lane;
      rv[u] = 0.0;
      if (pos < n) {
        const int t = perm[pos];
        int cp = 0;
#pragma unroll
        for (int c = 1; c < 8; ++c)
          if (t >= (int)eo[c] && es[c] >= 0) cp = c;
        rv[u] = __ldg(&r[es[cp] + (t - (int)eo[cp])]);
      }
    }
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int pos = p0 + u * 32 + lane;
      if (pos < n) y[pos] = (T)rv[u];
    }
  }
  __syncwarp();
  for (int l = 0; l < nlev; ++l) {
    const int v1 = lvl[l + 1];
    for (int v = lvl[l] + lane; v < v1; v += 32) {
      T acc = y[v];
      const int q1 = rowptr[v + 1];
      for (int q = rowptr[v]; q < q1; ++q) acc -= rowv[q] * y[rowidx[q]];
      y[v] = acc * invd[v];
    }
    __syncwarp();
  }
  for (int l = nlev - 1; l >= 0; --l) {
    const int v1 = lvl[l + 1];
    for (int v = lvl[l] + lane; v < v1; v += 32) {
      T acc = y[v];
      const int q1 = colptr[v + 1];
      for (int q = colptr[v]; q < q1; ++q) acc -= colv[q] * y[colidx[q]];
      y[v] = acc * invd[v];
    }
    __syncwarp();
  }
  for (int pos = lane; pos < n; pos += 32) w[base + perm[pos]] = (double)y[pos];
}

// block b solves stars blk[b] .. blk[b+1]-1; a block flagged "global" (one star
// too large for the budget) reads its section from global memory and keeps y
// in the global scratch
template <class T>
__global__ void __launch_bounds__(SOLVE_WPB * 32) k_star_solve(const int32_t* __restrict__ blk,
                                                                const uint8_t* __restrict__ blk_global,
                                                                const char* __restrict__ spool,
                                                                const int64_t* __restrict__ soff,
                                                                const int64_t* __restrict__ star_ptr,
                                                                const double* __restrict__ r,
                                                                double* __restrict__ w, T* ybuf,
                                                                const int* done) {
  extern __shared__ int4 smem4[];
  if (done && *done) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int s0 = blk[blockIdx.x], s1 = blk[blockIdx.x + 1];
  const int64_t g0 = soff[s0], g1 = soff[s1];
  if (blk_global[blockIdx.x]) {
    for (int s = s0 + wid; s < s1; s += SOLVE_WPB) {
      const char* sec = spool + soff[s];
      const int nnz = ((const int32_t*)sec)[2];
      T* y = ybuf + star_ptr[s];
      if (nnz > 65535) solve_section<T, uint32_t>(sec, y, r, w, lane);
      else solve_section<T, uint16_t>(sec, y, r, w, lane);
    }
    return;
  }
  const int n4 = (int)((g1 - g0) >> 4);
  const int4* src = (const int4*)(spool + g0);
  for (int q = threadIdx.x; q < n4; q += blockDim.x) smem4[q] = __ldg(&src[q]);
  __syncthreads();
  const char* sm = (const char*)smem4;
  for (int s = s0 + wid; s < s1; s += SOLVE_WPB) {
    // y of this star after all sections, behind the vectors of the block's earlier stars
    int64_t yo = g1 - g0;
    for (int t = s0; t < s; ++t) yo += align_up((int64_t)sizeof(T) * ((const int32_t*)(sm + (soff[t] - g0)))[0], 16);
    const char* sec = sm + (soff[s] - g0);
    const int nnz = ((const int32_t*)sec)[2];
    T* y = (T*)(sm + yo);
    if (nnz > 65535) solve_section<T, uint32_t>(sec, y, r, w, lane);
    else solve_section<T, uint16_t>(sec, y, r, w, lane);
  }
}

void launch_star_solve(spnet_pc_s* pc, const double* r, const int* done, cudaStream_t s) {
  if (pc->S == 0) return;
  note_launch();
  ProfScope ps(KID_STARS, s);
  if (pc->precision == SPNET_PREC_FP64)
    k_star_solve<double><<<pc->solve_blocks, SOLVE_WPB * 32, SOLVE_BUDGET, s>>>(
        pc->blk_star, pc->blk_global, pc->spool, pc->soff, pc->star_ptr, r, pc->w, (double*)pc->ybuf, done);
  else
    k_star_solve<float><<<pc->solve_blocks, SOLVE_WPB * 32, SOLVE_BUDGET, s>>>(
        pc->blk_star, pc->blk_global, pc->spool, pc->soff, pc->star_ptr, r, pc->w, (float*)pc->ybuf, done);
}

// compact sections in star order, grouped into blocks by the shared-memory budget
static int pack_sections(spnet_pc_s* pc, DevArena& tmp) {
  cudaStream_t s = pc->op->stream;
  const int S = pc->S;
  const int vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  int64_t* sz = nullptr;
  int32_t* yb = nullptr;
  SPNET_TRY(tmp.get(&sz, S + 1));
  SPNET_TRY(tmp.get(&yb, S));
  SPNET_TRY(pc->mem.get(&pc->soff, S + 1));
  note_launch();
  k_sec_sizes<<<(S + 255) / 256, 256, 0, s>>>(S, pc->pool, pc->star_off, vb, sz, yb);
  SPNET_TRY(scan_exclusive64(sz, pc->soff, S, s, tmp));
  std::vector<int64_t> hoff(S + 1);
  std::vector<int32_t> hyb(S);
  SPNET_CUDA_TRY(cudaMemcpyAsync(hoff.data(), pc->soff, sizeof(int64_t) * (S + 1), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaMemcpyAsync(hyb.data(), yb, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  pc->spool_bytes = hoff[S];
  SPNET_TRY(pc->mem.get(&pc->spool, hoff[S] > 0 ? hoff[S] : 16));
  note_launch();
  if (vb == 8)
    k_sec_pack<double><<<(S + 3) / 4, 128, 0, s>>>(S, mesh_of_pc(pc), pc->pool, pc->star_off, pc->star_mesh,
                                                   pc->elem_ptr, pc->star_ptr, pc->spool, pc->soff);
  else
    k_sec_pack<float><<<(S + 3) / 4, 128, 0, s>>>(S, mesh_of_pc(pc), pc->pool, pc->star_off, pc->star_mesh,
                                                  pc->elem_ptr, pc->star_ptr, pc->spool, pc->soff);
  // greedy grouping in star order
  std::vector<int32_t> blk;
  std::vector<uint8_t> glob;
  int st = 0;
  while (st < S) {
    int e = st;
    int64_t bytes = 0;
    while (e < S && e - st < SOLVE_WPB) {
      const int64_t add = (hoff[e + 1] - hoff[e]) + hyb[e];
      if (bytes + add > SOLVE_BUDGET) break;
      bytes += add;
      ++e;
    }
    blk.push_back(st);
    if (e == st) {  // one star beyond the budget: solved from global memory
      glob.push_back(1);
      e = st + 1;
    } else {
      glob.push_back(0);
    }
    st = e;
  }
  blk.push_back(S);
  pc->solve_blocks = (int)glob.size();
  SPNET_TRY(pc->mem.get(&pc->blk_star, blk.size()));
  SPNET_TRY(pc->mem.get(&pc->blk_global, glob.size()));
  SPNET_CUDA_TRY(cudaMemcpyAsync(pc->blk_star, blk.data(), sizeof(int32_t) * blk.size(), cudaMemcpyHostToDevice, s));
  SPNET_CUDA_TRY(cudaMemcpyAsync(pc->blk_global, glob.data(), glob.size(), cudaMemcpyHostToDevice, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  static bool attr_set[64][2] = {};
  int dev = 0;
  SPNET_CUDA_TRY(cudaGetDevice(&dev));
  dev &= 63;
  if (vb == 8 && !attr_set[dev][1]) {
    SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_BUDGET));
    attr_set[dev][1] = true;
  }
  if (vb == 4 && !attr_set[dev][0]) {
    SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_BUDGET));
    attr_set[dev][0] = true;
  }
  return SPNET_OK;
}

int pc_factor_stars(spnet_pc_s* pc) {
  cudaStream_t s = pc->op->stream;
  if (pc->S == 0) return SPNET_OK;
  if (pc->max_star > 65535)
    return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: a star holds more than 65535 dofs");
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const int nmax = pc->max_star;
  const int64_t hot = hot_bytes(nmax);
  // hot arrays in shared memory when four warps' worth fit in 200 KiB, one
  // block of four warps per SM at least; otherwise everything in global scratch
  const int hot_in_smem = 4 * hot <= 200 * 1024 ? 1 : 0;
  const int64_t stride = cold_bytes(nmax) + (hot_in_smem ? 0 : align_up(hot, 256));
  int wpb_blocks = hot_in_smem ? (int)((200 * 1024) / (4 * hot)) : 4;  // blocks per SM
  if (wpb_blocks < 1) wpb_blocks = 1;
  if (wpb_blocks > 4) wpb_blocks = 4;
  int64_t warps = (int64_t)4 * wpb_blocks * num_sms();
  int64_t budget = (int64_t)1 << 30;
  if (warps * stride > budget) warps = budget / stride;
  if (warps < 4) warps = 4;
  if (warps > pc->S) warps = pc->S;
  warps = (warps + 3) / 4 * 4;
  if (hot_in_smem) {
    static bool attr_set[64] = {};
    int dev = 0;
    SPNET_CUDA_TRY(cudaGetDevice(&dev));
    dev &= 63;
    if (!attr_set[dev]) {
      SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_symbolic, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr_set[dev] = true;
    }
  }
  char* scratch = nullptr;
  SPNET_TRY(tmp.get(&scratch, warps * stride));
  int* counters = nullptr;  // [0] next star, [2..3] pool top (u64)
  SPNET_TRY(tmp.get(&counters, 4));
  SPNET_TRY(pc->mem.get(&pc->star_off, pc->S));
  SPNET_TRY(pc->mem.get(&pc->star_lev, pc->S));
  SPNET_TRY(pc->mem.get(&pc->star_nnz, pc->S));
  // pool estimate: per dof 28 bytes + ~4 factor entries of 32 bytes, per star 64
  int64_t cap = pc->sum_s * (28 + 4 * 32) + (int64_t)pc->S * 64 + (1 << 20);
  int* flags = pc->op->dflags;
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (pc->pool) pc->mem.release(pc->pool);
    pc->pool = nullptr;
    SPNET_TRY(pc->mem.get(&pc->pool, cap));
    pc->pool_bytes = cap;
    SPNET_CUDA_TRY(cudaMemsetAsync(counters, 0, sizeof(int) * 4, s));
    SPNET_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
    StarArgs A;
    A.m = mesh_of_pc(pc);
    A.S = pc->S;
    A.star_mesh = pc->star_mesh;
    A.star_n = pc->star_n;
    A.elem_ptr = pc->elem_ptr;
    A.elem_of = pc->elem_of;
    A.kptr = pc->K.ptr;
    A.kcol = pc->K.col;
    A.kval = pc->K.val;
    A.scratch = scratch;
    A.stride = stride;
    A.hot = hot;
    A.hot_in_smem = hot_in_smem;
    A.nmax = nmax;
    A.pool = pc->pool;
    A.pool_cap = cap;
    A.pool_top = (unsigned long long*)(counters + 2);
    A.star_off = pc->star_off;
    A.star_lev = pc->star_lev;
    A.star_nnz = pc->star_nnz;
    A.flags = flags;
    A.next = counters;
    A.vbytes = 8;  // the set-up blobs keep FP64 values; the solve sections are packed later
    note_launch();
    ProfScope ps(KID_STAR_SYMBOLIC, s);
    k_star_symbolic<<<(unsigned)(warps / 4), 128, hot_in_smem ? (size_t)(4 * hot) : 0, s>>>(A);
    SPNET_CUDA_TRY(cudaGetLastError());
    int h = 0;
    SPNET_CUDA_TRY(cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));
    if (h & FLAG_POOL) {
      cap *= 3;
      continue;
    }
    if (h) return check_flags(flags, s, "setup_preconditioner (star structure)");
    break;
  }
  {
    int h = 0;
    SPNET_CUDA_TRY(cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return check_flags(flags, s, "setup_preconditioner (star pool)");
  }
  int blocks = (pc->S + 3) / 4;
  note_launch();
  ProfScope ps(KID_STAR_NUMERIC, s);
  k_star_numeric<<<blocks, 128, 0, s>>>(pc->S, pc->pool, pc->star_off, pc->K.ptr, pc->K.col,
                                         pc->K.val, 8, flags);
  SPNET_CUDA_TRY(cudaGetLastError());
  SPNET_TRY(check_flags(flags, s, "setup_preconditioner (star factorisation)"));
  // statistics
  std::vector<int32_t> lev(pc->S), nz(pc->S);
  SPNET_CUDA_TRY(cudaMemcpyAsync(lev.data(), pc->star_lev, sizeof(int32_t) * pc->S, cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaMemcpyAsync(nz.data(), pc->star_nnz, sizeof(int32_t) * pc->S, cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  pc->factor_nnz = 0;
  pc->total_levels = 0;
  pc->max_levels = 0;
  for (int i = 0; i < pc->S; ++i) {
    pc->factor_nnz += nz[i];
    pc->total_levels += lev[i];
    pc->max_levels = lev[i] > pc->max_levels ? lev[i] : pc->max_levels;
  }
  // vectors of stars solved from global memory, then the packed solve sections;
  // the set-up blobs are released
  const int vbytes = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  SPNET_TRY(pc->mem.alloc(&pc->ybuf, (size_t)pc->sum_s * vbytes));
  SPNET_TRY(pack_sections(pc, tmp));
  pc->mem.release(pc->pool);
  pc->pool = nullptr;
  return SPNET_OK;
}

}  // namespace spnet
