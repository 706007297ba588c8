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
  int64_t stride;  // scratch bytes per warp
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

__host__ __device__ inline int64_t scratch_bytes(int nmax) {
  int64_t o = 0;
  o += 2ll * nmax * CAP;
  o += 2ll * ((int64_t)nmax * CAP + CORE_ENTRIES);
  o = align_up(o, 8);
  o += 4ll * nmax * 2 + 4ll * (nmax + 1) * 5 + nmax;
  return align_up(o, 256);
}

__device__ inline Scratch carve(char* base, int nmax) {
  Scratch s;
  int64_t o = 0;
  s.nbr = (uint16_t*)(base + o);    o += 2ll * nmax * CAP;
  s.colent = (uint16_t*)(base + o); o += 2ll * ((int64_t)nmax * CAP + CORE_ENTRIES);
  o = align_up(o, 8);
  s.deg = (int32_t*)(base + o);      o += 4ll * nmax;
  s.state = (int32_t*)(base + o);    o += 4ll * nmax;
  s.posnode = (int32_t*)(base + o);  o += 4ll * (nmax + 1);
  s.colstart = (int32_t*)(base + o); o += 4ll * (nmax + 1);
  s.lvl = (int32_t*)(base + o);      o += 4ll * (nmax + 1);
  s.rcnt = (int32_t*)(base + o);     o += 4ll * (nmax + 1);
  s.rstart = (int32_t*)(base + o);   o += 4ll * (nmax + 1);
  s.sel = (uint8_t*)(base + o);
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
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const Scratch W = carve(A.scratch + wg * A.stride, A.nmax);
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

__global__ void k_solve_need(int S, const char* pool, const int64_t* star_off, int vbytes, int* mx) {
  int m = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const int32_t* hdr = (const int32_t*)(pool + star_off[s]);
    const BlobLayout L = blob_layout(hdr[0], hdr[1], hdr[2], vbytes);
    int need = (int)(L.solve + align_up((int64_t)vbytes * hdr[0], 16));
    m = max(m, need);
  }
  atomicMax(mx, m);
}

// ---------------------------------------------------------------------------
// the solve: gather r over the star, forward and backward level sweeps, write
// w_j in the star's element-concatenated order
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128) k_star_solve(int S, const char* __restrict__ pool,
                                                    const int64_t* __restrict__ star_off,
                                                    const int64_t* __restrict__ star_ptr,
                                                    const double* __restrict__ r, T* ybuf,
                                                    double* __restrict__ w, int spw, const int* done) {
  extern __shared__ __align__(16) char smem[];
  if (done && *done) return;
  const int lane = threadIdx.x & 31;
  char* mine = smem + (threadIdx.x >> 5) * spw;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nw) {
    const char* blob = pool + star_off[s];
    const int4 h = *(const int4*)blob;
    const int n = h.x, nlev = h.y, nnz = h.z;
    const BlobLayout L = blob_layout(n, nlev, nnz, (int)sizeof(T));
    const int64_t base = star_ptr[s];
    const char* src;
    T* y;
    if (L.solve + align_up((int64_t)sizeof(T) * n, 16) <= spw) {
      // stage the solve section in shared memory (16-byte vector copies)
      const int4* g4 = (const int4*)blob;
      int4* s4 = (int4*)mine;
      const int n4 = (int)(L.solve >> 4);
      for (int q = lane; q < n4; q += 32) s4[q] = __ldg(&g4[q]);
      src = mine;
      y = (T*)(mine + L.solve);
      __syncwarp();
    } else {
      src = blob;
      y = ybuf + base;
    }
    const int32_t* gidx = (const int32_t*)(src + L.gidx);
    const uint16_t* perm = (const uint16_t*)(src + L.perm);
    const uint16_t* lvl = (const uint16_t*)(src + L.lvl);
    const uint32_t* colptr = (const uint32_t*)(src + L.colptr);
    const uint16_t* colidx = (const uint16_t*)(src + L.colidx);
    const uint32_t* rowptr = (const uint32_t*)(src + L.rowptr);
    const uint16_t* rowidx = (const uint16_t*)(src + L.rowidx);
    const T* rowv = (const T*)(src + L.rowval);
    const T* colv = (const T*)(src + L.colval);
    const T* invd = (const T*)(src + L.invd);
    for (int pos = lane; pos < n; pos += 32) y[pos] = (T)r[gidx[pos]];
    __syncwarp();
    for (int l = 0; l < nlev; ++l) {
      for (int v = lvl[l] + lane; v < (int)lvl[l + 1]; v += 32) {
        T acc = y[v];
        for (uint32_t q = rowptr[v]; q < rowptr[v + 1]; ++q) acc -= rowv[q] * y[rowidx[q]];
        y[v] = acc * invd[v];
      }
      __syncwarp();
    }
    for (int l = nlev - 1; l >= 0; --l) {
      for (int v = lvl[l] + lane; v < (int)lvl[l + 1]; v += 32) {
        T acc = y[v];
        for (uint32_t q = colptr[v]; q < colptr[v + 1]; ++q) acc -= colv[q] * y[colidx[q]];
        y[v] = acc * invd[v];
      }
      __syncwarp();
    }
    for (int pos = lane; pos < n; pos += 32) w[base + perm[pos]] = (double)y[pos];
    __syncwarp();
  }
}

void launch_star_solve(spnet_pc_s* pc, const double* r, const int* done, cudaStream_t s) {
  if (pc->S == 0) return;
  const int wpb = 4;
  const int spw = pc->solve_spw;
  int blocks = (pc->S + wpb - 1) / wpb;
  note_launch();
  ProfScope ps(KID_STARS, s);
  if (pc->precision == SPNET_PREC_FP64)
    k_star_solve<double><<<blocks, 32 * wpb, (size_t)spw * wpb, s>>>(
        pc->S, pc->pool, pc->star_off, pc->star_ptr, r, (double*)pc->ybuf, pc->w, spw, done);
  else
    k_star_solve<float><<<blocks, 32 * wpb, (size_t)spw * wpb, s>>>(
        pc->S, pc->pool, pc->star_off, pc->star_ptr, r, (float*)pc->ybuf, pc->w, spw, done);
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
  const int64_t stride = scratch_bytes(nmax);
  // warps of the symbolic pass: bounded by the scratch budget (1 GiB) and by the star count
  int64_t warps = (int64_t)8 * num_sms();
  int64_t budget = (int64_t)1 << 30;
  if (warps * stride > budget) warps = budget / stride;
  if (warps < 4) warps = 4;
  if (warps > pc->S) warps = pc->S;
  warps = (warps + 3) / 4 * 4;
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
    A.nmax = nmax;
    A.pool = pc->pool;
    A.pool_cap = cap;
    A.pool_top = (unsigned long long*)(counters + 2);
    A.star_off = pc->star_off;
    A.star_lev = pc->star_lev;
    A.star_nnz = pc->star_nnz;
    A.flags = flags;
    A.next = counters;
    A.vbytes = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
    note_launch();
    ProfScope ps(KID_STAR_SYMBOLIC, s);
    k_star_symbolic<<<(unsigned)(warps / 4), 128, 0, s>>>(A);
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
  const int vbytes = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  k_star_numeric<<<blocks, 128, 0, s>>>(pc->S, pc->pool, pc->star_off, pc->K.ptr, pc->K.col,
                                         pc->K.val, vbytes, flags);
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
  // local solve buffers (used by stars that do not fit the shared-memory stage)
  SPNET_TRY(pc->mem.alloc(&pc->ybuf, (size_t)pc->sum_s * vbytes));
  // shared memory per warp: the largest star's solve section and vector, capped
  {
    int* mx = counters;
    SPNET_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(int), s));
    note_launch();
    k_solve_need<<<(pc->S + 255) / 256, 256, 0, s>>>(pc->S, pc->pool, pc->star_off, vbytes, mx);
    int need = 0;
    SPNET_CUDA_TRY(cudaMemcpyAsync(&need, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));
    const int cap = 48 * 1024;
    pc->solve_spw = (int)align_up(need < cap ? need : cap, 16);
    // the kernel attribute is process-wide: allow the largest stage any
    // preconditioner may ask for (4 warps x cap)
    static bool attr_set[64][2] = {};
    int dev = 0;
    SPNET_CUDA_TRY(cudaGetDevice(&dev));
    dev &= 63;
    const int bytes = 4 * cap;
    if (vbytes == 8 && !attr_set[dev][1]) {
      SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      attr_set[dev][1] = true;
    }
    if (vbytes == 4 && !attr_set[dev][0]) {
      SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
      attr_set[dev][0] = true;
    }
  }
  return SPNET_OK;
}

}  // namespace spnet
