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
#include <algorithm>
#include <climits>
#include <atomic>
#include <cmath>
#include <queue>
#include <tuple>
#include <mutex>
#include <map>

#include "spnet_internal.cuh"

namespace spnet {

// Adjacency slots per node during elimination: 32, or for matrices with longer rows
// (the beam model couples a node with its neighbours' neighbours, up to ~60 entries
// a row) three times as many as the longest row holds off the diagonal, rounded up to
// a multiple of 32 and at most 192.  The rest of a star turns dense once the minimum
// degree passes three quarters of the capacity.  With 32 slots a list that overflows
// turns the rest dense at once; with more, the node whose list overflows is frozen
// instead: it is kept for the dense block and the elimination goes on around it
// (its own list stays incomplete; every other list stays complete, and a fill pair
// is looked up in the list of a member that is not frozen).  On the beam model this
// shrinks the dense block of a 7,400-dof star from about 3,700 dofs to about 900.
constexpr int CAP_MIN = 32;
constexpr int CAP_MAX = 192;
__host__ __device__ inline int adjacency_cap(int max_offdiag) {
  if (max_offdiag <= 24) return CAP_MIN;
  int c = (3 * max_offdiag + 31) / 32 * 32;
  return c < CAP_MAX ? c : CAP_MAX;
}
constexpr int ST_FROZEN = -2;  // elimination state of a frozen node (alive: -1; eliminated: position)
__host__ __device__ inline int switch_degree(int cap) { return cap - cap / 4; }
constexpr int CORE_FIRST = 256;  // dense block capacity of the first attempt (raised 4x on overflow)

__host__ __device__ inline int64_t core_entries(int core_max) { return (int64_t)core_max * (core_max - 1) / 2; }

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
  int core_max;    // largest dense block the scratch holds
  char* pool;
  int64_t pool_cap;
  unsigned long long* pool_top;
  int64_t* star_off;
  int32_t* star_lev;
  int32_t* star_nnz;
  int32_t* star_core;
  int* flags;
  int* next;
  int vbytes;
  int cap;            // adjacency slots per node (adjacency_cap)
  int patch;          // SPNET_PATCH_*
  const double* q1w;  // [nc][N] Q1 values (the support rule tests them against zero)
  int64_t N;
};

struct Scratch {
  int cap;
  uint16_t* nbr;     // [nmax*cap]
  uint16_t* colent;  // [nmax*cap + core_entries(core_max)]
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
__host__ __device__ inline int64_t hot_bytes(int nmax, int cap) {
  return align_up(2ll * nmax * cap, 16) + align_up(8ll * nmax, 16) + align_up((int64_t)nmax, 16);
}

__host__ __device__ inline int64_t cold_bytes(int nmax, int core_max, int cap) {
  int64_t o = 2ll * ((int64_t)nmax * cap + core_entries(core_max));
  o = align_up(o, 8);
  o += 4ll * (nmax + 1) * 6;
  return align_up(o, 256);
}

__device__ inline Scratch carve(char* cold, char* hot, int nmax, int core_max, int cap) {
  Scratch s;
  s.cap = cap;
  int64_t o = 0;
  s.nbr = (uint16_t*)(hot + o);   o = align_up(o + 2ll * nmax * cap, 16);
  s.deg = (int32_t*)(hot + o);    o += 4ll * nmax;
  s.state = (int32_t*)(hot + o);  o = align_up(o + 4ll * nmax, 16);
  s.sel = (uint8_t*)(hot + o);
  o = 0;
  s.colent = (uint16_t*)(cold + o); o += 2ll * ((int64_t)nmax * cap + core_entries(core_max));
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

// "support" patches: local dof t lies outside the open support of the star's basis
// function (its Q1 value there is zero).  The star's mesh node sits at corner
// nc - 1 - c' of the element in slot c'.
__device__ inline bool off_support(const StarElems& se, const int32_t* elem_ptr, const double* q1w,
                                   int64_t N, int t) {
  int cp = 0;
  while (cp + 1 < se.nc && se.off[cp + 1] <= t) ++cp;
  const int i = elem_ptr[se.e[cp]] + (t - se.off[cp]);
  return q1w[(int64_t)(se.nc - 1 - cp) * N + i] == 0.0;
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

// remove the nodes eliminated by the current elimination step from the adjacency lists
// that hold them.
// Those are the lists of the round's column entries c0..c1 (the alive neighbours of the
// eliminated nodes; every other list holds alive nodes only), each marked once in sel
// (free after the round's selection) and compacted in order by the lane that meets it.
__device__ inline void compact_touched(const Scratch& W, int n, int lane, int c0, int c1) {
  for (int q = c0 + lane; q < c1; q += 32) W.sel[W.colent[q]] = 2;
  __syncwarp();
  for (int t = lane; t < n; t += 32) {
    if (W.sel[t] != 2) continue;
    W.sel[t] = 0;
    uint16_t* lst = W.nbr + (int64_t)t * W.cap;
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
  char* hot = A.hot_in_smem ? sm_hot + (threadIdx.x >> 5) * A.hot : cold + cold_bytes(A.nmax, A.core_max, A.cap);
  const Scratch W = carve(cold, hot, A.nmax, A.core_max, A.cap);
  const int CAP = A.cap, SWITCH_DEG = switch_degree(A.cap);
  const bool FREEZE = A.cap > CAP_MIN;
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
    // adjacency of the star graph (with support patches a dof off the support is an
    // isolated node: its row of the local matrix is the identity, and its solve
    // coefficient is zero, so the star adds nothing there)
    bool ovf = false;
    for (int t = lane; t < n; t += 32) {
      int i = pc_of_local(se, A.elem_ptr, t);
      int cnt = 0;
      bool o = false;
      const bool tex = A.patch == SPNET_PATCH_SUPPORT && off_support(se, A.elem_ptr, A.q1w, A.N, t);
      for (int64_t q = tex ? A.kptr[i + 1] : A.kptr[i]; q < A.kptr[i + 1]; ++q) {
        int j = A.kcol[q];
        if (j == i) continue;
        int lt = local_of_pc(A.m, se, A.elem_ptr, A.elem_of, km[0], km[1], km[2], j);
        if (lt < 0) continue;
        if (A.patch == SPNET_PATCH_SUPPORT && off_support(se, A.elem_ptr, A.q1w, A.N, lt)) continue;
        if (cnt < CAP) W.nbr[(int64_t)t * CAP + cnt++] = (uint16_t)lt;
        else o = true;
      }
      W.deg[t] = cnt;
      W.state[t] = o && FREEZE ? ST_FROZEN : -1;
      ovf |= o && !FREEZE;
    }
    ovf = __any_sync(FULL, ovf);
    __syncwarp();
    int npos = 0, nlev = 0, ncol = 0;
    bool dense = ovf;
    while (!dense && npos < n) {
      int md = 1 << 30;  // over the nodes that may still be eliminated
      for (int t = lane; t < n; t += 32)
        if (W.state[t] == -1) md = min(md, W.deg[t]);
      md = warp_min(md);
      if (md > SWITCH_DEG) {
        dense = true;
        break;
      }
      const int thr = max(md, 2);
      // independent set: candidates of degree <= thr that beat every candidate neighbour
      for (int t = lane; t < n; t += 32) {
        bool sl = false;
        if (W.state[t] == -1 && W.deg[t] <= thr) {
          sl = true;
          const int dt = W.deg[t];
          const uint16_t* lst = W.nbr + (int64_t)t * CAP;
          for (int q = 0; q < dt; ++q) {
            int u = lst[q];
            int du = W.deg[u];
            if (W.state[u] == -1 && du <= thr && (du < dt || (du == dt && u < t))) {
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
      compact_touched(W, n, lane, W.colstart[lev_start], ncol);
      // fill among the neighbours of each eliminated node: every pair (a, b) of
      // a column of this elimination step, 32 pairs at a time.  Lanes test adjacency in
      // parallel; pairs repeated inside a batch are merged; new list slots go
      // by rank among the lanes that extend the same list (deterministic).  A
      // list that would pass CAP entries switches the rest to the dense core.
      bool full = false;
      {
        int total = 0;  // pairs of the round; prefix per position in W.rstart
        for (int base = lev_start; base < npos; base += 32) {
          const int pos = base + lane;
          int c = 0;
          if (pos < npos) {
            const int d = W.colstart[pos + 1] - W.colstart[pos];
            c = d * (d - 1) / 2;
          }
          const int incl = warp_incl_scan(c, lane);
          if (pos < npos) W.rstart[pos - lev_start] = total + incl - c;
          total += __shfl_sync(FULL, incl, 31);
        }
        __syncwarp();
        const int nl = npos - lev_start;
        for (int p0 = 0; p0 < total; p0 += 32) {
          const int p = p0 + lane;
          int a = -1, b = -1;
          if (p < total) {
            int lo = 0, hi = nl - 1;  // position of pair p: last prefix <= p
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (W.rstart[mid] <= p) lo = mid;
              else hi = mid - 1;
            }
            const int pos = lev_start + lo;
            int l = p - W.rstart[lo];
            const int cs = W.colstart[pos], d = W.colstart[pos + 1] - cs;
            int ai = 0;
            while (l >= d - 1 - ai) {
              l -= d - 1 - ai;
              ++ai;
            }
            a = W.colent[cs + ai];
            b = W.colent[cs + ai + 1 + l];
            const bool fa = W.state[a] == ST_FROZEN, fb = W.state[b] == ST_FROZEN;
            if (fa && fb) {
              a = b = -1;  // both in the dense block, where every pair is coupled
            } else {
              const int c0 = fa ? b : a, c1 = fa ? a : b;  // look up in a complete list
              const int dc = W.deg[c0];
              bool found = false;
              for (int q = 0; q < dc; ++q) found |= W.nbr[(int64_t)c0 * CAP + q] == c1;
              if (found) a = b = -1;
            }
          }
          const unsigned key = a < 0 ? 0xffffffffu : ((unsigned)min(a, b) << 16) | (unsigned)max(a, b);
          const unsigned same = __match_any_sync(FULL, key);
          const bool ins = a >= 0 && __ffs(same) - 1 == lane;
#pragma unroll
          for (int side = 0; side < 2; ++side) {  // b into the list of a, then a into the list of b
            const int x = side == 0 ? a : b, y = side == 0 ? b : a;
            const bool insx = ins && W.state[x] != ST_FROZEN;  // a frozen list takes nothing more
            const unsigned grp = __match_any_sync(FULL, insx ? (unsigned)x : 0xffffffffu);
            const int rank = __popc(grp & ((1u << lane) - 1u));
            const int dx = insx ? W.deg[x] : 0;
            __syncwarp();
            if (insx) {
              if (dx + rank < CAP) W.nbr[(int64_t)x * CAP + dx + rank] = (uint16_t)y;
              else if (FREEZE) W.state[x] = ST_FROZEN;
              else full = true;
              if (rank == 0) W.deg[x] = min(dx + __popc(grp), CAP);
            }
            __syncwarp();
          }
        }
        full = __any_sync(FULL, full);
      }
      nlev++;
      if (full) dense = true;
    }
    if (dense && npos < n && A.patch == SPNET_PATCH_SUPPORT) {
      // dofs off the support still alive (all of them when the first adjacency
      // overflowed) are isolated: one level of their own ahead of the dense block,
      // so that the block couples none of them
      const int p0 = npos;
      for (int base = 0; base < n; base += 32) {
        int t = base + lane;
        bool al = t < n && W.state[t] < 0 && off_support(se, A.elem_ptr, A.q1w, A.N, t);
        unsigned b = __ballot_sync(FULL, al);
        if (al) {
          int pos = npos + __popc(b & ((1u << lane) - 1u));
          W.posnode[pos] = t;
          W.colstart[pos] = ncol;
          W.state[t] = pos;
        }
        npos += __popc(b);
      }
      if (npos > p0) {
        if (lane == 0) W.lvl[nlev] = p0;
        nlev++;
      }
      __syncwarp();
    }
    int core_c = 0;  // nodes of the dense block
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
      if (c > A.core_max || ncol + core_entries(c) > (int64_t)A.nmax * CAP + core_entries(A.core_max)) {
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
      core_c = c;
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
      A.star_core[s] = core_c;
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

// the longest row of K (entries), for the adjacency capacity
__global__ void k_max_row(int64_t n, const int64_t* __restrict__ ptr, int* out) {
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int)(ptr[i + 1] - ptr[i]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
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

// A group of TPS threads per star (a warp, four stars to a block; or the whole
// block of 128 when stars are large): a wide level gives a column to each
// thread, a narrow one (the dense block: one node per level) takes its columns
// in turn with their entries across the threads; a barrier ends each level.
constexpr int NT = 128;

template <int TPS>
__device__ __forceinline__ void group_sync() {
  if constexpr (TPS == 32) __syncwarp();
  else __syncthreads();
}

template <int TPS>
__global__ void __launch_bounds__(NT) k_star_numeric(int S, char* pool, const int64_t* star_off,
                                                     const int64_t* kptr, const int32_t* kcol,
                                                     const double* kval, int vbytes, int* flags) {
  constexpr int GPB = NT / TPS;  // stars per block at a time
  const int tid = threadIdx.x % TPS;
  for (int64_t s = (int64_t)blockIdx.x * GPB + threadIdx.x / TPS; s < S; s += (int64_t)gridDim.x * GPB) {
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
    // L_iv = (K_iv - sum_k L_vk L_ik) / L_vv for the entries of column v: a
    // merge of the sparse rows v and i (only earlier levels meet there)
    auto entries = [&](int v, int gv, double inv, uint32_t q0, uint32_t q1, uint32_t dq) {
      const uint32_t rv0 = rowptr[v], rv1 = rowptr[v + 1];
      for (uint32_t q = q0; q < q1; q += dq) {
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
    };
    auto pivot = [&](int v, int gv) {
      double d = k_entry(kptr, kcol, kval, gv, gv);
      for (uint32_t q = rowptr[v]; q < rowptr[v + 1]; ++q) d -= rowv[q] * rowv[q];
      if (!(d > 0.0)) {
        bad = true;
        d = 1.0;
      }
      return 1.0 / sqrt(d);
    };
    for (int l = 0; l < nlev; ++l) {
      const int v0 = lvl[l], v1 = lvl[l + 1];
      if (v1 - v0 >= 32) {  // a wide level: a column per thread
        for (int v = v0 + tid; v < v1; v += TPS) {
          const int gv = gidx[v];
          const double inv = pivot(v, gv);
          invd[v] = inv;
          entries(v, gv, inv, colptr[v], colptr[v + 1], 1);
        }
      } else {  // a narrow level: its columns in turn, their entries across the threads
        for (int v = v0; v < v1; ++v) {
          const int gv = gidx[v];
          const double inv = pivot(v, gv);  // every thread the same sum
          if (tid == 0) invd[v] = inv;
          entries(v, gv, inv, colptr[v] + tid, colptr[v + 1], TPS);
        }
      }
      group_sync<TPS>();
    }
    const bool any_bad = TPS == 32 ? __any_sync(0xffffffffu, bad) : __syncthreads_or(bad);
    if (any_bad && tid == 0) atomicOr(flags, FLAG_NOT_SPD);
    if (vbytes == 4) {
      float* r32 = (float*)(blob + L.rowval);
      for (int q = tid; q < 2 * nnz + n; q += TPS) r32[q] = (float)rowv[q];
    }
    group_sync<TPS>();
  }
}

// ---------------------------------------------------------------------------
// Solve windows.  Both triangular solves of a star are written as one sequence
// of entries (column, coefficient), level after level: the forward levels of
// L y = r in elimination order, then the levels of L^T z = y in reverse.  A row
// v of a level is a segment of consecutive entries
//   forward:   (u, -L_vu / L_vv) for the u of row v, then (v, 1 / L_vv)
//   backward:  (u, -L_uv / L_vv) for the u of column v, then (v, 1 / L_vv)
// so that the new value of row v is the segment's sum of coefficient *
// y[column], the diagonal entry last: its column names the row written.  Rows
// of one level do not read one another, so the sums of a level run in parallel
// and the update is in place.
//
// A level's entries are cut into windows of 32 slots (zero coefficients pad the
// last one; a padding slot reads y[0]).  Each window is one record:
//   descriptor (8 B): u32 mask of the slots that end a segment, u8 scan steps
//   (the longest segment inside the window needs that many doublings), u8 flags
//   (bit 0: the window's last segment continues in the next window); 8 B pad;
//   32 u16 columns; 32 coefficients in the solve precision.
// Everything that depends only on the factor is decided here, at set-up, so a
// window costs the solve a handful of instructions: one product per lane, a
// segmented shuffle scan of `steps` steps (a fixed order: deterministic), the
// writes of the segment ends, a carry of a cut segment into the next window.
//
// A warp solves one star.  Records stream through a ring of RING_W windows in
// shared memory (cp.async, one group per window); only the star's vector and
// its inverse permutation stay resident.
// ---------------------------------------------------------------------------
constexpr int WIN = 32;                      // slots per window
constexpr int RING_W = 16;                   // windows in flight
constexpr int STREAM_MAX_N = 65535;          // star size the u16 columns address
constexpr int STREAM_SMEM = 200 * 1024;      // shared memory budget per block
constexpr int REC_HDR = 16;                  // descriptor + pad
constexpr int REC_COEF = REC_HDR + 2 * WIN;  // offset of the coefficients

__host__ __device__ inline int rec_bytes(int vb) { return REC_COEF + WIN * vb; }  // 208 or 336

// per-star header of the solve, 80 bytes
struct StarHdr {
  int64_t eoff;   // first window record of the star
  int64_t wbase;  // first slot of the star in w (star_ptr)
  int32_t n;      // dofs
  int32_t ne;     // window records (forward + backward)
  int32_t es[8];  // pc index of the first dof of each of the 2^d elements, -1 if absent
  uint16_t eo[9]; // local offset of each element's dofs within the star
  uint16_t pad[3];
};
static_assert(sizeof(StarHdr) == 80, "StarHdr layout");

// Stars beyond LARGE_STAR dofs are solved by a variant that holds fewer bytes per
// warp in shared memory (an 8-window ring; the inverse permutation re-read from L2
// when the results are written), so that more warps stay resident.
constexpr int LARGE_STAR = 1024;
constexpr int RING_LARGE = 8;

// shared memory of one warp: ring, y, inverse permutation (not for large stars), header
__host__ __device__ inline int64_t stream_warp_bytes(int vb, int ymax, bool large = false) {
  return (int64_t)(large ? RING_LARGE : RING_W) * rec_bytes(vb) + align_up((int64_t)vb * ymax, 16) +
         (large ? 0 : align_up(2ll * ymax, 16)) + (int64_t)sizeof(StarHdr);
}

// windows of a level with E entries
__host__ __device__ inline int level_windows(int64_t E) { return (int)((E + WIN - 1) / WIN); }

// entries of level l: forward (row form) or backward (column form)
__device__ inline int64_t level_entries(const uint32_t* ptr, const uint16_t* lvl, int l) {
  const int v0 = lvl[l], v1 = lvl[l + 1];
  return (int64_t)(ptr[v1] - ptr[v0]) + (v1 - v0);
}

__global__ void k_stream_sizes(int S, const char* pool, const int64_t* star_off, int64_t* sz) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const char* blob = pool + star_off[s];
    const int32_t* h = (const int32_t*)blob;
    const int n = h[0], nlev = h[1], nnz = h[2];
    const BlobLayout B = blob_layout(n, nlev, nnz, 8);
    const uint32_t* rowptr = (const uint32_t*)(blob + B.rowptr);
    const uint32_t* colptr = (const uint32_t*)(blob + B.colptr);
    const uint16_t* lvl = (const uint16_t*)(blob + B.lvl);
    int64_t nw = 0;
    for (int l = 0; l < nlev; ++l)
      nw += level_windows(level_entries(rowptr, lvl, l)) + level_windows(level_entries(colptr, lvl, l));
    sz[s] = nw;
  }
}

// scan steps a window needs: a segment of at least 2^k + 1 slots holds 2^k
// consecutive slots that end no segment
__device__ inline int window_steps(unsigned ends, int cnt) {
  unsigned run = ~ends & (cnt >= 32 ? 0xffffffffu : ((1u << cnt) - 1u));
  int steps = 0;
  while (run) {
    run &= run >> (1 << steps);
    ++steps;
  }
  return steps;
}

// which elimination positions of a star lie off its basis function's support
struct SupportTest {
  int patch;
  StarElems se;
  const int32_t* elem_ptr;
  const double* q1w;
  int64_t N;
  const uint16_t* perm;  // elimination position -> local index
  __device__ bool off(int v) const {
    return patch == SPNET_PATCH_SUPPORT && off_support(se, elem_ptr, q1w, N, perm[v]);
  }
};

// the descriptor of every window of a level of E entries (ends set already): scan
// steps and the carry flag
__device__ inline void finish_level(char* recs, int64_t wb, int lane, int64_t E, int RB) {
  __syncwarp();
  __threadfence_block();
  const int nwl = level_windows(E);
  for (int k = lane; k < nwl; k += 32) {
    char* rec = recs + (wb + k) * RB;
    const int cnt = (int)((E - (int64_t)k * WIN) < WIN ? (E - (int64_t)k * WIN) : WIN);
    const unsigned ends = *(volatile unsigned*)rec;
    const int steps = window_steps(ends, cnt);
    const unsigned carry = (cnt == WIN && !((ends >> 31) & 1u)) ? 1u : 0u;
    ((unsigned*)rec)[1] = (unsigned)steps | (carry << 8);
  }
  __syncwarp();
}

// the windows of one level: entries of the rows of the level in order, the
// descriptor of every window (ends, steps, carry flag)
template <class T>
__device__ void pack_level(char* recs, int64_t wb, int lane, int v0, int v1, const uint32_t* ptr,
                           const uint16_t* idx, const double* val, const double* invd, int vb,
                           const SupportTest& sup) {
  const int RB = rec_bytes(vb);
  const int64_t E = (int64_t)(ptr[v1] - ptr[v0]) + (v1 - v0);
  for (int v = v0 + lane; v < v1; v += 32) {
    // a dof off the star's support (support patches) is an isolated row: a zero
    // coefficient makes its value, and the star's contribution there, zero
    const double dv = sup.off(v) ? 0.0 : invd[v];
    int64_t j = (int64_t)(ptr[v] - ptr[v0]) + (v - v0);
    for (uint32_t q = ptr[v]; q <= ptr[v + 1]; ++q, ++j) {
      const bool diag = q == ptr[v + 1];
      char* rec = recs + (wb + j / WIN) * RB;
      const int sl = (int)(j % WIN);
      ((uint16_t*)(rec + REC_HDR))[sl] = diag ? (uint16_t)v : idx[q];
      ((T*)(rec + REC_COEF))[sl] = (T)(diag ? dv : -val[q] * dv);
      if (diag) atomicOr((unsigned*)rec, 1u << sl);
    }
  }
  finish_level(recs, wb, lane, E, RB);
}

// warp per star: set-up blob (FP64 factor) -> header, inverse permutation, window records
template <class T>
__global__ void k_stream_pack(int S, Mesh m, const char* __restrict__ pool, const int64_t* __restrict__ star_off,
                              const int32_t* __restrict__ star_mesh, const int32_t* __restrict__ elem_ptr,
                              const int64_t* __restrict__ star_ptr, const int64_t* __restrict__ roff,
                              StarHdr* __restrict__ hdr, uint16_t* __restrict__ iperm, char* __restrict__ recs,
                              int patch, const double* __restrict__ q1w, int64_t N) {
  const int lane = threadIdx.x & 31;
  const int vb = (int)sizeof(T);
  const int RB = rec_bytes(vb);
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nw) {
    const char* blob = pool + star_off[s];
    const int32_t* hb = (const int32_t*)blob;
    const int n = hb[0], nlev = hb[1], nnz = hb[2];
    const BlobLayout B = blob_layout(n, nlev, nnz, 8);
    const uint32_t* rowptr = (const uint32_t*)(blob + B.rowptr);
    const uint32_t* colptr = (const uint32_t*)(blob + B.colptr);
    const uint16_t* lvl = (const uint16_t*)(blob + B.lvl);
    const uint16_t* perm = (const uint16_t*)(blob + B.perm);
    const uint16_t* rowidx = (const uint16_t*)(blob + B.rowidx);
    const uint16_t* colidx = (const uint16_t*)(blob + B.colidx);
    const double* rowv = (const double*)(blob + B.v64);
    const double* colv = rowv + nnz;
    const double* invd = colv + nnz;
    const int64_t r0 = roff[s], r1 = roff[s + 1], wb = star_ptr[s];
    if (lane == 0) {
      StarHdr h;
      h.eoff = r0;
      h.wbase = wb;
      h.n = n;
      h.ne = (int32_t)(r1 - r0);
      const StarElems se = star_elems(m, star_mesh[s], elem_ptr);
      for (int cp = 0; cp < 8; ++cp) h.es[cp] = (cp < m.nc && se.e[cp] >= 0) ? elem_ptr[se.e[cp]] : -1;
      for (int cp = 0; cp <= 8; ++cp) h.eo[cp] = (uint16_t)(cp <= m.nc ? se.off[cp < m.nc ? cp : m.nc] : n);
      h.pad[0] = h.pad[1] = h.pad[2] = 0;
      hdr[s] = h;
    }
    for (int pos = lane; pos < n; pos += 32) iperm[wb + perm[pos]] = (uint16_t)pos;
    // zero records (padding slots: column 0, coefficient 0)
    int4* z4 = (int4*)(recs + r0 * RB);
    const int64_t n16 = (r1 - r0) * RB / 16;
    for (int64_t q = lane; q < n16; q += 32) z4[q] = make_int4(0, 0, 0, 0);
    __syncwarp();
    __threadfence_block();
    SupportTest sup;
    sup.patch = patch;
    sup.se = star_elems(m, star_mesh[s], elem_ptr);
    sup.elem_ptr = elem_ptr;
    sup.q1w = q1w;
    sup.N = N;
    sup.perm = perm;
    int64_t w = r0;
    for (int l = 0; l < nlev; ++l) {  // forward levels
      pack_level<T>(recs, w, lane, lvl[l], lvl[l + 1], rowptr, rowidx, rowv, invd, vb, sup);
      w += level_windows(level_entries(rowptr, lvl, l));
    }
    for (int l = nlev - 1; l >= 0; --l) {  // backward levels, last first
      pack_level<T>(recs, w, lane, lvl[l], lvl[l + 1], colptr, colidx, colv, invd, vb, sup);
      w += level_windows(level_entries(colptr, lvl, l));
    }
  }
}


// one scan step of the segmented inclusive scan: lanes at least o past their
// segment's first lane add the value o lanes down
template <class T>
__device__ __forceinline__ T scan_step(T v, int o, int dl) {
  const T t = __shfl_up_sync(0xffffffffu, v, o);
  return dl >= o ? v + t : v;
}

// slot (block, warp) -> star: sorder[blockIdx.x * wpb + warp], -1 for an idle slot.
// With q set (a PCG step) the right-hand side is the new residual r - alpha q
// (alpha from the SpMV), formed exactly as the update forms it; otherwise r.
template <class T, bool LARGE>
__global__ void __launch_bounds__(256) k_star_stream(int wpb, int ymax, const int32_t* __restrict__ sorder,
                                                     const StarHdr* __restrict__ hdr, const char* __restrict__ recs,
                                                     const uint16_t* __restrict__ iperm, const double* __restrict__ r,
                                                     const double* __restrict__ q, const Scal* sc,
                                                     T* __restrict__ w, const int* done) {
  extern __shared__ int4 smem4[];
  pdl_wait();
  pdl_trigger();
  if (done && *done) return;
  const double alpha = q ? sc->alpha : 0.0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int s = sorder[blockIdx.x * wpb + wid];
  if (s < 0) return;  // no block-wide barrier follows
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int RB = REC_COEF + WIN * (int)sizeof(T);
  constexpr int RW = LARGE ? RING_LARGE : RING_W;  // windows in flight
  constexpr unsigned RING_BYTES = (unsigned)(RW * RB);
  char* ring = (char*)smem4 + (int64_t)wid * stream_warp_bytes((int)sizeof(T), ymax, LARGE);
  T* y = (T*)(ring + RING_BYTES);
  uint16_t* ip = (uint16_t*)((char*)y + align_up((int64_t)sizeof(T) * ymax, 16));
  StarHdr* h = (StarHdr*)((char*)ip + (LARGE ? 0 : align_up(2ll * ymax, 16)));
  if (lane < (int)(sizeof(StarHdr) / 4)) ((int32_t*)h)[lane] = __ldg(((const int32_t*)(hdr + s)) + lane);
  __syncwarp();
  const int64_t wb = h->wbase;
  const int n = h->n, nw = h->ne;
  // records stream in order: src is the next record to fetch, dst its ring slot
  const bool copier = lane * 16 < RB;
  const char* src = recs + h->eoff * RB + lane * 16;
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  unsigned dst = ring_s + lane * 16;
  int F = 0;
  for (; F < nw && F < RW; ++F) {
    if (copier) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    src += RB;
    dst += RB;
  }
  if (dst - ring_s - lane * 16 >= RING_BYTES) dst -= RING_BYTES;
  // gather r over the star in local order (element ranges: coalesced), place it at the elimination position
  int eo[8], es[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    eo[c] = h->eo[c];
    es[c] = h->es[c];
  }
  constexpr int GU = 4;
  for (int t0 = 0; t0 < n; t0 += 32 * GU) {
    double rv[GU];
    int pv[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int t = t0 + u * 32 + lane;
      rv[u] = 0.0;
      pv[u] = 0;
      if (t < n) {
        int base = es[0] - eo[0];
#pragma unroll
        for (int c = 1; c < 8; ++c) base = t >= eo[c] ? es[c] - eo[c] : base;
        rv[u] = q ? fma(-alpha, __ldg(&q[base + t]), __ldg(&r[base + t])) : __ldg(&r[base + t]);
        pv[u] = __ldg(&iperm[wb + t]);
      }
    }
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int t = t0 + u * 32 + lane;
      if (t < n) {
        y[pv[u]] = (T)rv[u];
        if (!LARGE) ip[t] = (uint16_t)pv[u];
      }
    }
  }
  const unsigned le = FULL >> (31 - lane);  // lanes 0..lane
  const char* rec = ring;
  const char* const ring_end = ring + RING_BYTES;
  T carry = T(0);
  for (int k = 0; k < nw; ++k) {
    if (F == k + RW) asm volatile("cp.async.wait_group %0;\n" ::"n"(RW - 1) : "memory");
    else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    const uint2 d = *(const uint2*)rec;
    const int col = ((const uint16_t*)(rec + REC_HDR))[lane];
    const T a = ((const T*)(rec + REC_COEF))[lane];
    const unsigned ends = d.x;
    const unsigned steps = d.y & 0xffu;
    T v = a * y[col];
    const int dl = lane - (31 - __clz(((ends << 1) | 1u) & le));  // lanes since the segment's first
    if (steps > 0u) v = scan_step(v, 1, dl);
    if (steps > 1u) v = scan_step(v, 2, dl);
    if (steps > 2u) v = scan_step(v, 4, dl);
    if (steps > 3u) v = scan_step(v, 8, dl);
    if (steps > 4u) v = scan_step(v, 16, dl);
    // a segment cut by the previous window: its partial sum joins this window's first segment
    if (lane <= dl) v += carry;  // lanes of the first segment (dl == lane there)
    if ((ends >> lane) & 1u) y[col] = v;
    carry = T(0);
    if (d.y & 0x100u) carry = __shfl_sync(FULL, v, 31);
    __syncwarp();
    rec += RB;
    if (rec == ring_end) rec = ring;
    if (F < nw) {  // refill the slot just consumed
      if (copier) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      src += RB;
      dst += RB;
      if (dst - ring_s - lane * 16 >= RING_BYTES) dst -= RING_BYTES;
      ++F;
    }
  }
  for (int t = lane; t < n; t += 32) w[wb + t] = y[LARGE ? __ldg(&iperm[wb + t]) : ip[t]];
}

void launch_star_solve(spnet_pc_s* pc, const double* r, const double* q, const Scal* sc, const int* done,
                       cudaStream_t s) {
  if (pc->S == 0) return;
  note_launch();
  ProfScope ps(KID_STARS, s);
  const int wpb = pc->solve_wpb;
  const unsigned grid = (unsigned)pc->solve_blocks;
  const bool large = pc->max_star > LARGE_STAR;
  const StarHdr* hdr = (const StarHdr*)pc->shdr;
  if (pc->precision == SPNET_PREC_FP64) {
    auto kern = large ? k_star_stream<double, true> : k_star_stream<double, false>;
    kern<<<grid, wpb * 32, pc->solve_smem, s>>>(wpb, pc->max_star, pc->sorder, hdr, pc->srec, pc->iperm_star, r, q,
                                                sc, (double*)pc->w, done);
  } else {
    auto kern = large ? k_star_stream<float, true> : k_star_stream<float, false>;
    kern<<<grid, wpb * 32, pc->solve_smem, s>>>(wpb, pc->max_star, pc->sorder, hdr, pc->srec, pc->iperm_star, r, q,
                                                sc, (float*)pc->w, done);
  }
}

// ---------------------------------------------------------------------------
// Dense blocks with many right-hand sides, on tensor cores.
// The elimination of a large star ends in a dense block of c nodes, one node
// per level; such blocks hold most of the factor of large stars (over 80 % on
// the 200000-fibre 3D network and on the largest 2D serving requests) and,
// solved level by level, are a chain of 2c dependent steps.  In the k-right-
// hand-side solve (FP32) a star whose block has at least CORE_TC nodes runs
//   the forward sparse levels,
//   one level that removes the terms outside the block from the block's rows
//     (y_c = r_c - L_cn y_n),
//   L_cc y_c = y_c and L_cc^T z_c = y_c by panels of 16 rows,
//   the backward sparse levels.
// A forward panel step multiplies the panel by the inverse of its 16 x 16
// diagonal tile and subtracts L_rp y_p from every later panel r; a backward
// step uses the transposed tiles and updates the earlier panels.  Every
// product is a warp-level tensor-core MMA (m16n8k8 with TF32 inputs, each
// input split into a high and a low TF32 part and three products accumulated
// in FP32, which keeps FP32 accuracy).  The chain shrinks to 2 ceil(c/16)
// panel steps.
// A star's block area in coreL (floats), 16 x 16 blocks of 256 floats in MMA
// A-fragment order ([k half][lane][4]: lane l, value e holds row l/4 + 8 (e&1),
// column 8 khalf + l%4 + 4 (e>>1)), np = ceil(c / 16) panels:
//   DI(p), DIT(p)    inverse of diagonal tile p and its transpose
//   F(r, q), FT(r, q)  tile (r, q) of L_cc (r > q) and its transpose
// Rows and columns past c are zero.
// ---------------------------------------------------------------------------
constexpr int CORE_TC = 32;  // smallest dense block solved by panels

struct BatchHdr {
  int64_t eoff;   // first window record (in brec for a star solved with its block by panels, else srec)
  int64_t coff;   // first float of the star's block area in coreL (-1: none)
  int32_t nfwd;   // records before the block's solve
  int32_t ne;     // records in all
  int32_t core0;  // elimination position of the block's first node
  int32_t c;      // nodes of the block (0: no panel solve)
};
static_assert(sizeof(BatchHdr) == 32, "BatchHdr layout");

__host__ __device__ inline int core_panels(int c) { return (c + 15) / 16; }
__host__ __device__ inline int64_t core_floats(int c) {
  const int64_t np = core_panels(c);
  return 256 * np * (np + 1);
}
__host__ __device__ inline int64_t blk_DI(int p) { return 256ll * p; }
__host__ __device__ inline int64_t blk_DIT(int np, int p) { return 256ll * (np + p); }
__host__ __device__ inline int64_t blk_F(int np, int r, int q) { return 256ll * (2ll * np + (int64_t)r * (r - 1) / 2 + q); }
__host__ __device__ inline int64_t blk_FT(int np, int r, int q) {
  return 256ll * (2ll * np + (int64_t)np * (np - 1) / 2 + (int64_t)r * (r - 1) / 2 + q);
}

__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragments of rows rb .. rb+15 of the block's part of y (columns 0..7; columns past
// JW and rows past c read as zero), split into high and low TF32 parts: [k half][b0, b1]
struct PanelB {
  uint32_t h[2][2], l[2][2];
};
template <int JW>
__device__ __forceinline__ PanelB load_panel_b(const float* y, int core0, int rb, int c) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  PanelB B;
#pragma unroll
  for (int kh = 0; kh < 2; ++kh)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int r = rb + kh * 8 + t + 4 * e;
      const float v = (g < JW && r < c) ? y[(core0 + r) * JW + g] : 0.f;
      B.h[kh][e] = tf32_of(v);
      B.l[kh][e] = tf32_of(v - __uint_as_float(B.h[kh][e]));
    }
  return B;
}

// the A fragment of one k half, split into high and low TF32 parts
__device__ __forceinline__ void split_a(const float4 a, uint32_t (&ah)[4], uint32_t (&al)[4]) {
  const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    ah[e] = tf32_of(av[e]);
    al[e] = tf32_of(av[e] - __uint_as_float(ah[e]));
  }
}

// d[i] = block i (16 x 16, fragments at blk[i]) x the panel B, for NB blocks at once: their
// fragments are loaded together and their products interleaved (independent chains)
template <int NB>
__device__ __forceinline__ void blocks_mma(float (&d)[NB][4], const float* const (&blk)[NB], const PanelB& B) {
  const int lane = threadIdx.x & 31;
  float4 a[NB][2];
#pragma unroll
  for (int i = 0; i < NB; ++i)
#pragma unroll
    for (int kh = 0; kh < 2; ++kh) a[i][kh] = __ldg(reinterpret_cast<const float4*>(blk[i]) + kh * 32 + lane);
#pragma unroll
  for (int i = 0; i < NB; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) d[i][e] = 0.f;
#pragma unroll
  for (int kh = 0; kh < 2; ++kh) {
    uint32_t ah[NB][4], al[NB][4];
#pragma unroll
    for (int i = 0; i < NB; ++i) split_a(a[i][kh], ah[i], al[i]);
#pragma unroll
    for (int i = 0; i < NB; ++i) mma_tf32(d[i], al[i], B.h[kh][0], B.h[kh][1]);
#pragma unroll
    for (int i = 0; i < NB; ++i) mma_tf32(d[i], ah[i], B.l[kh][0], B.l[kh][1]);
#pragma unroll
    for (int i = 0; i < NB; ++i) mma_tf32(d[i], ah[i], B.h[kh][0], B.h[kh][1]);
  }
}

// rows rb + l/4 (+ 8), columns 2 (l%4) (+ 1) of the block's part of y: set (sub = false)
// or subtract (sub = true) the accumulator d
template <int JW>
__device__ __forceinline__ void blk_store(const float (&d)[4], float* y, int core0, int rb, int c, bool sub) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int row = rb + g + ((e >> 1) << 3), col = 2 * t + (e & 1);
    if (col < JW && row < c) {
      float* p = &y[(core0 + row) * JW + col];
      *p = sub ? *p - d[e] : d[e];
    }
  }
}

// subtract (block of panel r) x B from panel r, for the panels r of [r0, r1) (step dr), four
// at a time; blk(r) gives the block's fragments
template <int JW, class BlkOf>
__device__ __forceinline__ void panel_updates(const PanelB& B, float* y, int core0, int c, int r0, int r1,
                                              BlkOf blk) {
  int r = r0;
  for (; r + 4 <= r1; r += 4) {
    const float* const bl[4] = {blk(r), blk(r + 1), blk(r + 2), blk(r + 3)};
    float u[4][4];
    blocks_mma<4>(u, bl, B);
#pragma unroll
    for (int i = 0; i < 4; ++i) blk_store<JW>(u[i], y, core0, 16 * (r + i), c, true);
  }
  for (; r < r1; ++r) {
    const float* const bl[1] = {blk(r)};
    float u[1][4];
    blocks_mma<1>(u, bl, B);
    blk_store<JW>(u[0], y, core0, 16 * r, c, true);
  }
}

// L_cc y_c = y_c, then L_cc^T z_c = y_c, in place on the block's part of y (one warp)
template <int JW>
__device__ void core_panel_solve(const float* __restrict__ L, float* y, int core0, int c) {
  const int np = core_panels(c);
  for (int p = 0; p < np; ++p) {
    {
      const PanelB B = load_panel_b<JW>(y, core0, 16 * p, c);
      const float* const bl[1] = {L + blk_DI(p)};
      float d[1][4];
      blocks_mma<1>(d, bl, B);
      __syncwarp();
      blk_store<JW>(d[0], y, core0, 16 * p, c, false);
      __syncwarp();
    }
    const PanelB B = load_panel_b<JW>(y, core0, 16 * p, c);
    panel_updates<JW>(B, y, core0, c, p + 1, np, [&](int r) { return L + blk_F(np, r, p); });
    __syncwarp();
  }
  for (int p = np - 1; p >= 0; --p) {
    {
      const PanelB B = load_panel_b<JW>(y, core0, 16 * p, c);
      const float* const bl[1] = {L + blk_DIT(np, p)};
      float d[1][4];
      blocks_mma<1>(d, bl, B);
      __syncwarp();
      blk_store<JW>(d[0], y, core0, 16 * p, c, false);
      __syncwarp();
    }
    const PanelB B = load_panel_b<JW>(y, core0, 16 * p, c);
    panel_updates<JW>(B, y, core0, c, 0, p, [&](int r) { return L + blk_FT(np, p, r); });
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Star solves for k right-hand sides at once (k <= 32).  Each star is solved
// by kp / JW warps (kp: k rounded up to a power of two; JW = min(kp, 4)), one
// warp per block, each owning JW right-hand sides.  A warp streams the same
// window records as the one-right-hand-side solve; its lanes are (slot group
// q, right-hand side j): lane (q, j) sums slots q*JW .. q*JW + JW - 1 of each
// window for column j, a segmented scan over the 32 / JW groups (shuffles)
// joins the parts of a segment cut by a group boundary, and the sum of a
// segment still open at the window's end is carried into the next window.
// A window holds rows of one level only, so none of its slots reads a value
// the window writes: all its values are loaded before any sum is stored.
// The right-hand sides do not interact, the factor bytes are read from L2 by
// the kp / JW warps of a star together, and the sums of a column do not depend
// on the other columns or on k (for a given JW).
// R, W: [dofs][k] (right-hand side fastest); y in shared memory [n][JW].
// ---------------------------------------------------------------------------
constexpr int BRING = 8;  // windows in flight per warp

// right-hand sides per warp: 4 (measured on the 40000-fibre workload with 32
// right-hand sides: 89 ms of star solves against 110 ms with 8 and 118 ms with 2)
__host__ __device__ inline int batch_jw(int kp) { return kp < 4 ? kp : 4; }

__host__ __device__ inline int64_t batch_warp_bytes(int vb, int ymax, int jw) {
  return (int64_t)BRING * rec_bytes(vb) + align_up((int64_t)vb * ymax * jw, 16) + align_up(2ll * ymax, 16) +
         (int64_t)sizeof(StarHdr);
}

// the column indices of slots s0 .. s0 + SPL - 1 of a record (one vector load)
template <int SPL>
__device__ __forceinline__ void load_cols(const char* rec, int s0, int (&c)[SPL]) {
  const char* p = rec + REC_HDR + 2 * s0;
  if constexpr (SPL == 8) {
    const uint4 v = *(const uint4*)p;
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c[2 * i] = (int)(w[i] & 0xffffu);
      c[2 * i + 1] = (int)(w[i] >> 16);
    }
  } else if constexpr (SPL == 4) {
    const uint2 v = *(const uint2*)p;
    c[0] = (int)(v.x & 0xffffu);
    c[1] = (int)(v.x >> 16);
    c[2] = (int)(v.y & 0xffffu);
    c[3] = (int)(v.y >> 16);
  } else if constexpr (SPL == 2) {
    const unsigned v = *(const unsigned*)p;
    c[0] = (int)(v & 0xffffu);
    c[1] = (int)(v >> 16);
  } else {
    c[0] = *(const uint16_t*)p;
  }
}

// their coefficients (vector loads)
template <int SPL>
__device__ __forceinline__ void load_coefs(const char* rec, int s0, float (&a)[SPL]) {
  const float* p = (const float*)(rec + REC_COEF) + s0;
  if constexpr (SPL >= 4) {
#pragma unroll
    for (int i = 0; i < SPL / 4; ++i) {
      const float4 v = ((const float4*)p)[i];
      a[4 * i] = v.x;
      a[4 * i + 1] = v.y;
      a[4 * i + 2] = v.z;
      a[4 * i + 3] = v.w;
    }
  } else if constexpr (SPL == 2) {
    const float2 v = *(const float2*)p;
    a[0] = v.x;
    a[1] = v.y;
  } else {
    a[0] = p[0];
  }
}

template <int SPL>
__device__ __forceinline__ void load_coefs(const char* rec, int s0, double (&a)[SPL]) {
  const double* p = (const double*)(rec + REC_COEF) + s0;
  if constexpr (SPL >= 2) {
#pragma unroll
    for (int i = 0; i < SPL / 2; ++i) {
      const double2 v = ((const double2*)p)[i];
      a[2 * i] = v.x;
      a[2 * i + 1] = v.y;
    }
  } else {
    a[0] = p[0];
  }
}

template <class T, int JW>
__global__ void __launch_bounds__(32) k_star_batch(int k, int groups, int ymax, const int32_t* __restrict__ order,
                                                   const StarHdr* __restrict__ hdr, const char* __restrict__ recs,
                                                   const uint16_t* __restrict__ iperm,
                                                   const double* __restrict__ R, T* __restrict__ W,
                                                   const int* done, const BatchHdr* __restrict__ bhdr,
                                                   const char* __restrict__ brec, const float* __restrict__ coreL) {
  constexpr int QN = 32 / JW;    // slot groups of a window
  constexpr int SPL = WIN / QN;  // slots per lane (= JW)
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ int4 smem4[];
  pdl_wait();
  pdl_trigger();
  if (done && *done) return;
  const int lane = threadIdx.x;
  const int q = lane / JW, j = lane % JW;
  const int s = order[blockIdx.x / groups];
  const int jj = (blockIdx.x % groups) * JW + j;  // this lane's right-hand side
  const bool act = jj < k;
  constexpr int RB = REC_COEF + WIN * (int)sizeof(T);
  constexpr unsigned RING_BYTES = (unsigned)(BRING * RB);
  char* ring = (char*)smem4;
  T* y = (T*)(ring + RING_BYTES);
  uint16_t* ip = (uint16_t*)((char*)y + align_up((int64_t)sizeof(T) * ymax * JW, 16));
  StarHdr* h = (StarHdr*)((char*)ip + align_up(2ll * ymax, 16));
  if (lane < (int)(sizeof(StarHdr) / 4)) ((int32_t*)h)[lane] = __ldg(((const int32_t*)(hdr + s)) + lane);
  __syncwarp();
  const int64_t wb = h->wbase;
  const int n = h->n;
  int nw = h->ne, nfwd = h->ne, core0 = 0, cc = 0;
  int64_t eoff = h->eoff, coff = 0;
  const char* rbase = recs;
  if (bhdr) {  // a dense block solved by panels: its own record stream
    const BatchHdr bh = bhdr[s];
    if (bh.c > 0) {
      eoff = bh.eoff;
      nw = bh.ne;
      nfwd = bh.nfwd;
      core0 = bh.core0;
      cc = bh.c;
      coff = bh.coff;
      rbase = brec;
    }
  }
  const bool copier = lane * 16 < RB;
  const char* src = rbase + eoff * RB + lane * 16;
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  unsigned dst = ring_s + lane * 16;
  int F = 0;
  for (; F < nw && F < BRING; ++F) {
    if (copier) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    src += RB;
    dst += RB;
  }
  if (dst - ring_s - lane * 16 >= RING_BYTES) dst -= RING_BYTES;
  int eo[8], es[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    eo[c] = h->eo[c];
    es[c] = h->es[c];
  }
  // gather: y[position][j] = R[pc index][jj]; the lanes of a slot group take one local dof
  constexpr int GU = 16;
  for (int t0 = 0; t0 < n; t0 += QN * GU) {
    double rv[GU];
    int pv[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int t = t0 + u * QN + q;
      rv[u] = 0.0;
      pv[u] = 0;
      if (t < n) {
        int base = es[0] - eo[0];
#pragma unroll
        for (int c = 1; c < 8; ++c) base = t >= eo[c] ? es[c] - eo[c] : base;
        pv[u] = __ldg(&iperm[wb + t]);
        if (act) rv[u] = __ldg(&R[(int64_t)(base + t) * k + jj]);
      }
    }
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int t = t0 + u * QN + q;
      if (t < n) {
        y[pv[u] * JW + j] = (T)rv[u];  // right-hand sides past k hold zeros
        if (j == 0) ip[t] = (uint16_t)pv[u];
      }
    }
  }
  __syncwarp();
  const char* rec = ring;
  const char* const ring_end = ring + RING_BYTES;
  const int s0 = q * SPL;
  T carry = T(0);  // the open segment's sum from the previous window (column j)
  for (int w = 0; w < nw; ++w) {
    if constexpr (sizeof(T) == 4) {
      if (cc > 0 && w == nfwd) core_panel_solve<JW>(coreL + coff, (float*)y, core0, cc);
    }
    if (F == w + BRING) asm volatile("cp.async.wait_group %0;\n" ::"n"(BRING - 1) : "memory");
    else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    const uint2 d = *(const uint2*)rec;
    int c[SPL];
    T a[SPL], yv[SPL];
    load_cols<SPL>(rec, s0, c);
    load_coefs<SPL>(rec, s0, a);
#pragma unroll
    for (int i = 0; i < SPL; ++i) yv[i] = y[c[i] * JW + j];
    // this group's slots: segments that start and end here are stored at once
    T acc = T(0), head = T(0);
    int hc = -1;
#pragma unroll
    for (int i = 0; i < SPL; ++i) {
      acc = fma(a[i], yv[i], acc);
      if ((d.x >> (s0 + i)) & 1u) {
        if (hc < 0) {
          head = acc;  // the group's first segment end: the segment may have begun earlier
          hc = c[i];
        } else {
          y[c[i] * JW + j] = acc;
        }
        acc = T(0);
      }
    }
    // inclusive segmented scan over the groups: v = the open sum leaving group q
    T v = acc;
    int f = hc >= 0;
#pragma unroll
    for (int dd = 1; dd < QN; dd <<= 1) {
      const T ov = __shfl_up_sync(FULL, v, dd * JW);
      const int of = __shfl_up_sync(FULL, f, dd * JW);
      if (q >= dd) {
        if (!f) v += ov;
        f |= of;
      }
    }
    T vin = __shfl_up_sync(FULL, v, JW);
    int fin = __shfl_up_sync(FULL, f, JW);
    if (q == 0) {
      vin = T(0);
      fin = 0;
    }
    if (hc >= 0) y[hc * JW + j] = (fin ? vin : vin + carry) + head;
    const T vl = __shfl_sync(FULL, v, (QN - 1) * JW + j);
    const int fl = __shfl_sync(FULL, f, (QN - 1) * JW + j);
    carry = (d.y & 0x100u) ? (fl ? vl : vl + carry) : T(0);
    __syncwarp();
    rec += RB;
    if (rec == ring_end) rec = ring;
    if (F < nw) {  // refill the slot just consumed
      if (copier) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      src += RB;
      dst += RB;
      if (dst - ring_s - lane * 16 >= RING_BYTES) dst -= RING_BYTES;
      ++F;
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (cc > 0 && nfwd == nw) core_panel_solve<JW>(coreL + coff, (float*)y, core0, cc);
  }
  __syncwarp();
  if (act)
    for (int t = q; t < n; t += QN) W[(wb + t) * k + jj] = y[ip[t] * JW + j];
}

int star_batch_max_k(const spnet_pc_s* pc) {
  const int vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  int kp = 32;
  while (kp > 1 && batch_warp_bytes(vb, pc->max_star, batch_jw(kp)) > 227 * 1024) kp >>= 1;
  return kp;
}

template <class T, int JW>
static int star_batch_t(spnet_pc_s* pc, const double* R, int k, int kp, T* W, const int* done, cudaStream_t s) {
  const size_t smem = (size_t)batch_warp_bytes((int)sizeof(T), pc->max_star, JW);
  if (smem > 227 * 1024)
    return fail(SPNET_ERR_UNSUPPORTED, "star solves: the largest star's solve vector for " + std::to_string(k) +
                                           " right-hand sides exceeds a block's shared memory");
  static std::atomic<bool> attr_set[64];  // per device
  int dev = 0;
  SPNET_CUDA_TRY(cudaGetDevice(&dev));
  dev &= 63;
  if (!attr_set[dev]) {
    SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_batch<T, JW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr_set[dev] = true;
  }
  const int groups = kp / JW;
  const bool panels = sizeof(T) == 4 && pc->bhdr != nullptr;
  launch_pdl(k_star_batch<T, JW>, (unsigned)(pc->S * groups), 32, smem, s, k, groups, pc->max_star,
             (const int32_t*)pc->star_desc, (const StarHdr*)pc->shdr, (const char*)pc->srec,
             (const uint16_t*)pc->iperm_star, R, W, done, panels ? (const BatchHdr*)pc->bhdr : nullptr,
             panels ? (const char*)pc->brec : nullptr, panels ? (const float*)pc->coreL : nullptr);
  return SPNET_OK;
}

// Right-hand sides per warp: batch_jw.  (Eight per warp, a whole MMA width, halves the
// warps that replay a star's sparse records but doubles the shared memory of each: on
// the 200000-fibre network with 32 right-hand sides 74 against 52 ms per solve.)
template <class T>
static int star_batch_p(spnet_pc_s* pc, const double* R, int k, int kp, T* W, const int* done, cudaStream_t s) {
  int jw = batch_jw(kp);
  if (pc->batch_jw > 0 && pc->batch_jw < jw) jw = pc->batch_jw;  // the tuned width
  switch (jw) {
    case 1: return star_batch_t<T, 1>(pc, R, k, kp, W, done, s);
    case 2: return star_batch_t<T, 2>(pc, R, k, kp, W, done, s);
    default: return star_batch_t<T, 4>(pc, R, k, kp, W, done, s);
  }
}

int launch_star_batch(spnet_pc_s* pc, const double* R, int k, void* W, const int* done, cudaStream_t s) {
  if (pc->S == 0) return SPNET_OK;
  if (k < 1 || k > 32) return fail(SPNET_ERR_BAD_INPUT, "star solves: 1..32 right-hand sides at once");
  const int kp = k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
  note_launch();
  ProfScope ps(KID_STARS, s);
  if (pc->precision == SPNET_PREC_FP64) return star_batch_p<double>(pc, R, k, kp, (double*)W, done, s);
  return star_batch_p<float>(pc, R, k, kp, (float*)W, done, s);
}

// The star solve's mapping for `wpb` warps per block.  The solve is bound by
// the instruction issue of each SM, so every SM gets the same number k of
// blocks (a grid of k * SMs blocks; the shared memory of a block is padded so
// that no SM can hold more than k when they all fit in one wave) and the stars
// are dealt to the blocks largest first, each to the block with the least work
// so far.  Work of a star ~ entries / 32 + 2 levels.
static int build_star_map(spnet_pc_s* pc, int wpb) {
  cudaStream_t s = pc->op->stream;
  const int S = pc->S;
  const int vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  const bool large = pc->max_star > LARGE_STAR;
  const int64_t wb = stream_warp_bytes(vb, pc->max_star, large);
  const int nsm = num_sms();
  int k = (int)((S + (int64_t)nsm * wpb - 1) / ((int64_t)nsm * wpb));
  if (k < 1) k = 1;
  size_t smem = (size_t)(wpb * wb);
  auto occupancy = [&](size_t bytes, int* nb) -> cudaError_t {
    if (vb == 8)
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          nb, large ? k_star_stream<double, true> : k_star_stream<double, false>, wpb * 32, bytes);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        nb, large ? k_star_stream<float, true> : k_star_stream<float, false>, wpb * 32, bytes);
  };
  int nb = 0;
  SPNET_CUDA_TRY(occupancy(smem, &nb));
  if (nb >= k) {
    while (nb > k && smem + 1024 <= (size_t)STREAM_SMEM) {
      smem += 1024;
      SPNET_CUDA_TRY(occupancy(smem, &nb));
    }
    if (nb < k) smem -= 1024;  // never fewer than k blocks per SM
  }
  const int B = nsm * k;
  std::vector<int32_t> slot((size_t)B * wpb, -1);
  std::vector<int> fill(B, 0);
  std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>, std::greater<std::pair<double, int>>> heap;
  for (int b = 0; b < B; ++b) heap.push({0.0, b});
  for (int i : pc->star_ord) {
    const std::pair<double, int> top = heap.top();
    heap.pop();
    const int b = top.second;
    slot[(size_t)b * wpb + fill[b]++] = i;
    if (fill[b] < wpb) heap.push({top.first + pc->star_cost[i], b});
  }
  if (pc->sorder) {
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));  // no launch reads the old map any more
    pc->mem.release(pc->sorder);
    pc->sorder = nullptr;
  }
  SPNET_TRY(pc->mem.get(&pc->sorder, slot.size()));
  SPNET_CUDA_TRY(cudaMemcpyAsync(pc->sorder, slot.data(), sizeof(int32_t) * slot.size(), cudaMemcpyHostToDevice, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));  // the host slot table goes out of scope
  pc->solve_wpb = wpb;
  pc->solve_blocks = B;
  pc->solve_smem = smem;
  return SPNET_OK;
}

// Size class of the star solve: the solve precision, half-octaves of the star count, the
// largest star and the stream bytes per star (the tuner's cache keeps the warps per block
// timed best for each, per device).
static TuneClass map_class(const spnet_pc_s* pc) {
  const int vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  return TuneClass{{vb, half_octave(pc->S), half_octave(pc->max_star), half_octave((double)pc->stream_bytes / pc->S)}};
}

// the mapping to build first: the fixed one, the one cached for the size class, else the widest
static int initial_wpb(const spnet_pc_s* pc, int wmax) {
  if (pc->star_map > 0) return pc->star_map < wmax ? pc->star_map : wmax;
  int v = 0;
  if (pc->S == 0 || !tune_peek(TUNE_STAR_MAP, map_class(pc), &v)) return wmax;
  return v < wmax ? v : wmax;
}

int star_map_tune(spnet_pc_s* pc) {
  if (pc->S == 0 || pc->star_map > 0) return SPNET_OK;  // fixed: built so by pack_streams
  // fewer stars than four per SM: one wave holds them whatever the mapping
  if (pc->S < 4 * num_sms()) return SPNET_OK;
  const int wmax = pc->solve_wpb_max;
  const TuneClass key = map_class(pc);
  {
    int v = 0;
    if (tune_begin(TUNE_STAR_MAP, key, &v)) {  // known
      const int w = v < wmax ? v : wmax;
      if (w != pc->solve_wpb) SPNET_TRY(build_star_map(pc, w));
      return SPNET_OK;
    }
  }
  // candidates: the most warps per block the shared memory holds, half and a quarter of it
  std::vector<int> cand;
  for (int w = wmax; w >= 1 && (int)cand.size() < 3; w /= 2) cand.push_back(w);
  cudaStream_t s = pc->op->stream;
  SPNET_CUDA_TRY(cudaMemsetAsync(pc->vtmp, 0, sizeof(double) * pc->N, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SPNET_CUDA_TRY(cudaEventCreate(&e0));
  SPNET_CUDA_TRY(cudaEventCreate(&e1));
  // In a PCG step the star solve runs beside the update and the coarse product, where many
  // small blocks crowd those out: a narrower mapping is taken only when the solve is long
  // (200 us or more, where it sets the step's length) and beats the widest by 5 % alone.
  int best = wmax;
  float best_ms = 0.0f, wide_ms = 0.0f;
  int rc = SPNET_OK;
  for (int w : cand) {
    if ((rc = build_star_map(pc, w)) != SPNET_OK) break;
    launch_star_solve(pc, pc->vtmp, nullptr, nullptr, nullptr, s);  // warm-up
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3; ++rep) launch_star_solve(pc, pc->vtmp, nullptr, nullptr, nullptr, s);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = fail(SPNET_ERR_CUDA, "setup_preconditioner: timing the star solve failed");
      break;
    }
    if (w == cand.front()) {
      wide_ms = best_ms = ms;
      if (ms / 3.0f < 0.2f) break;  // a short solve: the widest mapping
    } else if (ms < best_ms && ms < 0.95f * wide_ms) {
      best = w;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tune_end(TUNE_STAR_MAP, key, rc == SPNET_OK ? best : 0);
  if (rc != SPNET_OK) return rc;
  if (best != pc->solve_wpb) SPNET_TRY(build_star_map(pc, best));
  return SPNET_OK;
}

// Right-hand sides per warp of the batched star solve (2 or 4), timed once per size class
// (precision and block width, half-octaves of the star count and the largest star, whether
// dense blocks are solved by panels) on the preconditioner's own stars, for the block
// width the preconditioner steps (batch_rhs).  The choice changes the order of the sums,
// so every set-up of a class takes the one measured value.
int batch_jw_tune(spnet_pc_s* pc) {
  pc->batch_jw = 0;
  const int k = pc->batch_rhs < 32 ? pc->batch_rhs : 32;
  if (pc->S == 0 || k < 4 || star_batch_max_k(pc) < 4) return SPNET_OK;
  const int kp = k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
  const int vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  const TuneClass key{{vb * 64 + kp, half_octave(pc->S), half_octave(pc->max_star), pc->panel_stars > 0 ? 1 : 0}};
  int v = 0;
  if (tune_begin(TUNE_BATCH_JW, key, &v)) {
    pc->batch_jw = v;
    return SPNET_OK;
  }
  cudaStream_t s = pc->op->stream;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const int64_t rbytes = 8ll * pc->N * k, wbytes = (int64_t)vb * pc->sum_s * k;
  int best = 4, rc = SPNET_OK;
  if (rbytes + wbytes > (2ll << 30)) {  // too large to time on the side: the default
    tune_end(TUNE_BATCH_JW, key, best);
    pc->batch_jw = best;
    return SPNET_OK;
  }
  double* R = nullptr;
  void* W = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((rc = tmp.get(&R, (size_t)pc->N * k)) || (rc = tmp.alloc(&W, (size_t)wbytes)) ||
      cudaMemsetAsync(R, 0, (size_t)rbytes, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    tune_end(TUNE_BATCH_JW, key, 0);
    return rc ? rc : fail(SPNET_ERR_CUDA, "setup_preconditioner: timing the batched star solve failed");
  }
  float best_ms = 0.0f;
  for (int jw : {4, 2}) {
    pc->batch_jw = jw;
    rc = launch_star_batch(pc, R, k, W, nullptr, s);  // warm-up
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 2 && rc == SPNET_OK; ++rep) rc = launch_star_batch(pc, R, k, W, nullptr, s);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (rc != SPNET_OK || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      if (rc == SPNET_OK) rc = fail(SPNET_ERR_CUDA, "setup_preconditioner: timing the batched star solve failed");
      break;
    }
    if (jw == 4 || ms < 0.95f * best_ms) {  // the narrower one must beat four per warp by 5 %
      best = jw;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tune_end(TUNE_BATCH_JW, key, rc == SPNET_OK ? best : 0);
  pc->batch_jw = rc == SPNET_OK ? best : 0;
  return rc;
}

// ---------------------------------------------------------------------------
// Set-up of the panel solves (see "Dense blocks with many right-hand sides")
// ---------------------------------------------------------------------------
// entries of the pre-update level: the block's rows, their entries outside the
// block (the first entries of each row) and a unit diagonal
__device__ inline int64_t pre_entries(const uint32_t* rowptr, int core0, int n) {
  const int64_t c = n - core0;
  return (int64_t)(rowptr[n] - rowptr[core0]) - c * (c - 1) / 2 + c;
}

// records of the k-right-hand-side stream and floats of the block area, per star
__global__ void k_panel_sizes(int S, const char* pool, const int64_t* star_off, const int32_t* star_core,
                              int64_t* nrec, int64_t* nflt) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const int c = star_core[s];
    if (c < CORE_TC) {
      nrec[s] = 0;
      nflt[s] = 0;
      continue;
    }
    const char* blob = pool + star_off[s];
    const int32_t* h = (const int32_t*)blob;
    const int n = h[0], nlev = h[1], nnz = h[2];
    const BlobLayout B = blob_layout(n, nlev, nnz, 8);
    const uint32_t* rowptr = (const uint32_t*)(blob + B.rowptr);
    const uint32_t* colptr = (const uint32_t*)(blob + B.colptr);
    const uint16_t* lvl = (const uint16_t*)(blob + B.lvl);
    int64_t nw = level_windows(pre_entries(rowptr, n - c, n));
    for (int l = 0; l < nlev - c; ++l)
      nw += level_windows(level_entries(rowptr, lvl, l)) + level_windows(level_entries(colptr, lvl, l));
    nrec[s] = nw;
    nflt[s] = core_floats(c);
  }
}

// the pre-update level: row v of the block gets y_v - sum over its columns u outside the
// block of L_vu y_u (a unit diagonal, coefficients -L_vu)
template <class T>
__device__ void pack_pre_level(char* recs, int64_t wb, int lane, int core0, int n, const uint32_t* rowptr,
                               const uint16_t* rowidx, const double* rowv, int vb) {
  const int RB = rec_bytes(vb);
  for (int v = core0 + lane; v < n; v += 32) {
    const int64_t i = v - core0;
    const uint32_t q1 = rowptr[v + 1] - (uint32_t)i;  // the block's own columns are the last i entries
    int64_t j = (int64_t)(rowptr[v] - rowptr[core0]) - i * (i - 1) / 2 + i;
    for (uint32_t q = rowptr[v]; q <= q1; ++q, ++j) {
      const bool diag = q == q1;
      char* rec = recs + (wb + j / WIN) * RB;
      const int sl = (int)(j % WIN);
      ((uint16_t*)(rec + REC_HDR))[sl] = diag ? (uint16_t)v : rowidx[q];
      ((T*)(rec + REC_COEF))[sl] = (T)(diag ? 1.0 : -rowv[q]);
      if (diag) atomicOr((unsigned*)rec, 1u << sl);
    }
  }
  finish_level(recs, wb, lane, pre_entries(rowptr, core0, n), RB);
}

// warp per star: the k-right-hand-side header, and for a star with a panel-solved block its
// records (forward sparse levels, pre-update level, backward sparse levels)
template <class T>
__global__ void k_panel_pack(int S, Mesh m, const char* __restrict__ pool, const int64_t* __restrict__ star_off,
                             const int32_t* __restrict__ star_core, const int32_t* __restrict__ star_mesh,
                             const int32_t* __restrict__ elem_ptr, const StarHdr* __restrict__ hdr,
                             const int64_t* __restrict__ boff, const int64_t* __restrict__ coff,
                             BatchHdr* __restrict__ bhdr, char* __restrict__ recs, int patch,
                             const double* __restrict__ q1w, int64_t N) {
  const int lane = threadIdx.x & 31;
  const int vb = (int)sizeof(T);
  const int RB = rec_bytes(vb);
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nwarps) {
    const int c = star_core[s];
    if (c < CORE_TC) {
      if (lane == 0) {
        BatchHdr b;
        b.eoff = hdr[s].eoff;
        b.coff = -1;
        b.nfwd = hdr[s].ne;
        b.ne = hdr[s].ne;
        b.core0 = hdr[s].n;
        b.c = 0;
        bhdr[s] = b;
      }
      continue;
    }
    const char* blob = pool + star_off[s];
    const int32_t* hb = (const int32_t*)blob;
    const int n = hb[0], nlev = hb[1], nnz = hb[2];
    const BlobLayout B = blob_layout(n, nlev, nnz, 8);
    const uint32_t* rowptr = (const uint32_t*)(blob + B.rowptr);
    const uint32_t* colptr = (const uint32_t*)(blob + B.colptr);
    const uint16_t* lvl = (const uint16_t*)(blob + B.lvl);
    const uint16_t* rowidx = (const uint16_t*)(blob + B.rowidx);
    const uint16_t* colidx = (const uint16_t*)(blob + B.colidx);
    const double* rowv = (const double*)(blob + B.v64);
    const double* colv = rowv + nnz;
    const double* invd = colv + nnz;
    const int core0 = n - c, lnc = nlev - c;
    const int64_t r0 = boff[s], r1 = boff[s + 1];
    int4* z4 = (int4*)(recs + r0 * RB);
    const int64_t n16 = (r1 - r0) * RB / 16;
    for (int64_t q = lane; q < n16; q += 32) z4[q] = make_int4(0, 0, 0, 0);
    __syncwarp();
    __threadfence_block();
    SupportTest sup;  // as in the one-vector stream
    sup.patch = patch;
    sup.se = star_elems(m, star_mesh[s], elem_ptr);
    sup.elem_ptr = elem_ptr;
    sup.q1w = q1w;
    sup.N = N;
    sup.perm = (const uint16_t*)(blob + B.perm);
    int64_t w = r0;
    for (int l = 0; l < lnc; ++l) {
      pack_level<T>(recs, w, lane, lvl[l], lvl[l + 1], rowptr, rowidx, rowv, invd, vb, sup);
      w += level_windows(level_entries(rowptr, lvl, l));
    }
    pack_pre_level<T>(recs, w, lane, core0, n, rowptr, rowidx, rowv, vb);
    w += level_windows(pre_entries(rowptr, core0, n));
    const int nfwd = (int)(w - r0);
    for (int l = lnc - 1; l >= 0; --l) {
      pack_level<T>(recs, w, lane, lvl[l], lvl[l + 1], colptr, colidx, colv, invd, vb, sup);
      w += level_windows(level_entries(colptr, lvl, l));
    }
    if (lane == 0) {
      BatchHdr b;
      b.eoff = r0;
      b.coff = coff[s];
      b.nfwd = nfwd;
      b.ne = (int32_t)(r1 - r0);
      b.core0 = core0;
      b.c = c;
      bhdr[s] = b;
    }
  }
}

// entry (a, b), a > b, of the block L_cc (local indices): row core0 + a lists the block's
// columns 0..a-1 as its last a entries
__device__ __forceinline__ double core_L(const uint32_t* rowptr, const double* rowv, int core0, int a, int b) {
  return rowv[rowptr[core0 + a + 1] - a + b];
}

// (inverse of the diagonal tile of panel p)[i][j], local i, j in 0..15 (zero past c):
// forward substitution on column j of the tile, in FP64
__device__ double diag_tile_inverse(const uint32_t* rowptr, const double* rowv, const double* invd, int core0,
                                    int c, int p, int i, int j) {
  const int r0 = 16 * p;
  if (i < j || r0 + i >= c || r0 + j >= c) return 0.0;
  double x[16];
  x[j] = invd[core0 + r0 + j];
  for (int m = j + 1; m <= i; ++m) {
    double acc = 0.0;
    for (int q = j; q < m; ++q) acc += core_L(rowptr, rowv, core0, r0 + m, r0 + q) * x[q];
    x[m] = -acc * invd[core0 + r0 + m];
  }
  return x[i];
}

// block per star with a panel-solved block: its block area in coreL (FP32)
__global__ void __launch_bounds__(256) k_core_pack(int S, const char* __restrict__ pool,
                                                   const int64_t* __restrict__ star_off,
                                                   const int32_t* __restrict__ star_core,
                                                   const int64_t* __restrict__ coff, float* __restrict__ coreL) {
  for (int s = blockIdx.x; s < S; s += gridDim.x) {
    const int c = star_core[s];
    if (c < CORE_TC) continue;
    const char* blob = pool + star_off[s];
    const int32_t* hb = (const int32_t*)blob;
    const int n = hb[0], nlev = hb[1], nnz = hb[2];
    const BlobLayout B = blob_layout(n, nlev, nnz, 8);
    const uint32_t* rowptr = (const uint32_t*)(blob + B.rowptr);
    const double* rowv = (const double*)(blob + B.v64);
    const double* invd = rowv + 2ll * nnz;
    const int core0 = n - c, np = core_panels(c);
    float* out = coreL + coff[s];
    const int64_t total = core_floats(c);
    for (int64_t f = threadIdx.x; f < total; f += blockDim.x) {
      const int64_t blk = f >> 8;
      const int in = (int)(f & 255);
      const int kh = in >> 7, ln = (in >> 2) & 31, e = in & 3;
      const int li = (ln >> 2) + ((e & 1) << 3);       // row inside the 16 x 16 block
      const int lj = kh * 8 + (ln & 3) + ((e >> 1) << 2);  // column inside it
      double v = 0.0;
      if (blk < np) {  // DI(p)
        v = diag_tile_inverse(rowptr, rowv, invd, core0, c, (int)blk, li, lj);
      } else if (blk < 2 * np) {  // DIT(p)
        v = diag_tile_inverse(rowptr, rowv, invd, core0, c, (int)(blk - np), lj, li);
      } else {
        int64_t t = blk - 2 * np;
        const int64_t half = (int64_t)np * (np - 1) / 2;
        const bool tr = t >= half;
        if (tr) t -= half;
        int r = 1;
        while ((int64_t)r * (r + 1) / 2 <= t) ++r;  // t = r (r - 1) / 2 + q
        const int q = (int)(t - (int64_t)r * (r - 1) / 2);
        // F(r, q)[li][lj] = L_cc[16 r + li][16 q + lj]; FT(r, q)[li][lj] = L_cc[16 r + lj][16 q + li]
        const int a = tr ? 16 * r + lj : 16 * r + li;
        const int b = tr ? 16 * q + li : 16 * q + lj;
        if (a < c && b < c) v = core_L(rowptr, rowv, core0, a, b);
      }
      out[f] = (float)v;
    }
  }
}

// the k-right-hand-side stream and block areas (FP32 solves with batch_rhs >= 2)
static int pack_panels(spnet_pc_s* pc, DevArena& tmp) {
  cudaStream_t s = pc->op->stream;
  const int S = pc->S;
  std::vector<int32_t> core(S);
  SPNET_CUDA_TRY(cudaMemcpyAsync(core.data(), pc->star_core, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  int dense = 0;
  for (int v : core) dense += v >= CORE_TC;
  pc->panel_stars = dense;
  if (dense == 0) return SPNET_OK;
  int64_t *nrec = nullptr, *nflt = nullptr, *boff = nullptr, *coff = nullptr;
  SPNET_TRY(tmp.get(&nrec, S + 1));
  SPNET_TRY(tmp.get(&nflt, S + 1));
  SPNET_TRY(tmp.get(&boff, S + 1));
  SPNET_TRY(tmp.get(&coff, S + 1));
  note_launch();
  k_panel_sizes<<<(S + 255) / 256, 256, 0, s>>>(S, pc->pool, pc->star_off, pc->star_core, nrec, nflt);
  SPNET_TRY(scan_exclusive64(nrec, boff, S, s, tmp));
  SPNET_TRY(scan_exclusive64(nflt, coff, S, s, tmp));
  int64_t tr = 0, tf = 0;
  SPNET_CUDA_TRY(cudaMemcpyAsync(&tr, boff + S, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaMemcpyAsync(&tf, coff + S, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  const int RB = rec_bytes(4);
  SPNET_TRY(pc->mem.alloc(&pc->bhdr, (size_t)S * sizeof(BatchHdr)));
  SPNET_TRY(pc->mem.get(&pc->brec, (tr > 0 ? tr : 1) * RB));
  SPNET_TRY(pc->mem.get(&pc->coreL, tf > 0 ? tf : 1));
  pc->panel_bytes = tr * RB + tf * 4;
  note_launch();
  k_panel_pack<float><<<(S + 3) / 4, 128, 0, s>>>(S, mesh_of_pc(pc), pc->pool, pc->star_off, pc->star_core,
                                                  pc->star_mesh, pc->elem_ptr, (const StarHdr*)pc->shdr, boff, coff,
                                                  (BatchHdr*)pc->bhdr, pc->brec, pc->star_rule, pc->patch_w, pc->N);
  note_launch();
  const int grid = S < 8 * num_sms() ? S : 8 * num_sms();
  k_core_pack<<<grid, 256, 0, s>>>(S, pc->pool, pc->star_off, pc->star_core, coff, pc->coreL);
  SPNET_CUDA_TRY(cudaGetLastError());
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  return SPNET_OK;
}

// headers, inverse permutations and entry streams of all stars
static int pack_streams(spnet_pc_s* pc, DevArena& tmp, const std::vector<int32_t>& lev,
                        const std::vector<int32_t>& nz) {
  cudaStream_t s = pc->op->stream;
  const int S = pc->S;
  const int vb = pc->precision == SPNET_PREC_FP64 ? 8 : 4;
  int64_t* sz = nullptr;
  int64_t* roff = nullptr;
  SPNET_TRY(tmp.get(&sz, S + 1));
  SPNET_TRY(tmp.get(&roff, S + 1));
  note_launch();
  k_stream_sizes<<<(S + 255) / 256, 256, 0, s>>>(S, pc->pool, pc->star_off, sz);
  SPNET_TRY(scan_exclusive64(sz, roff, S, s, tmp));
  int64_t total = 0;
  SPNET_CUDA_TRY(cudaMemcpyAsync(&total, roff + S, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  const int RB = rec_bytes(vb);
  pc->n_entries = total;  // window records
  SPNET_TRY(pc->mem.alloc(&pc->shdr, (size_t)S * sizeof(StarHdr)));
  SPNET_TRY(pc->mem.get(&pc->iperm_star, pc->sum_s > 0 ? pc->sum_s : 1));
  SPNET_TRY(pc->mem.get(&pc->srec, (total > 0 ? total : 1) * RB));
  pc->stream_bytes = (int64_t)S * (int64_t)sizeof(StarHdr) + 2 * pc->sum_s + (int64_t)RB * total;
  note_launch();
  if (vb == 8)
    k_stream_pack<double><<<(S + 3) / 4, 128, 0, s>>>(S, mesh_of_pc(pc), pc->pool, pc->star_off, pc->star_mesh,
                                                      pc->elem_ptr, pc->star_ptr, roff, (StarHdr*)pc->shdr,
                                                      pc->iperm_star, pc->srec, pc->star_rule, pc->patch_w, pc->N);
  else
    k_stream_pack<float><<<(S + 3) / 4, 128, 0, s>>>(S, mesh_of_pc(pc), pc->pool, pc->star_off, pc->star_mesh,
                                                     pc->elem_ptr, pc->star_ptr, roff, (StarHdr*)pc->shdr,
                                                     pc->iperm_star, pc->srec, pc->star_rule, pc->patch_w, pc->N);
  SPNET_CUDA_TRY(cudaGetLastError());
  // warps per block: as many as the shared-memory budget holds, at most eight
  const int64_t wb = stream_warp_bytes(vb, pc->max_star, pc->max_star > LARGE_STAR);
  int wpb = (int)(STREAM_SMEM / wb);
  wpb = wpb > 8 ? 8 : wpb;
  if (wpb < 1) return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: a star too large for the solve's shared memory");
  static std::atomic<bool> attr_set[64][2];  // per device and precision (workers may race: setting twice is harmless)
  int dev = 0;
  SPNET_CUDA_TRY(cudaGetDevice(&dev));
  dev &= 63;
  if (vb == 8 && !attr_set[dev][1]) {
    SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_stream<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, STREAM_SMEM));
    SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_stream<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, STREAM_SMEM));
    attr_set[dev][1] = true;
  }
  if (vb == 4 && !attr_set[dev][0]) {
    SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_stream<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, STREAM_SMEM));
    SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_stream<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, STREAM_SMEM));
    attr_set[dev][0] = true;
  }
  std::vector<int32_t> sn(S);
  SPNET_CUDA_TRY(cudaMemcpyAsync(sn.data(), pc->star_n, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  pc->star_cost.assign(S, 0.0);
  pc->star_ord.resize(S);
  for (int i = 0; i < S; ++i) {
    pc->star_cost[i] = 2.0 * ((double)sn[i] + nz[i]) / 32.0 + 2.0 * lev[i];
    pc->star_ord[i] = i;
  }
  const std::vector<double>& cost = pc->star_cost;
  std::stable_sort(pc->star_ord.begin(), pc->star_ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  SPNET_TRY(pc->mem.get(&pc->star_desc, S));  // stars by cost, largest first (multi-right-hand-side solves)
  SPNET_CUDA_TRY(cudaMemcpyAsync(pc->star_desc, pc->star_ord.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
  pc->solve_wpb_max = wpb;
  SPNET_TRY(build_star_map(pc, initial_wpb(pc, wpb)));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  return SPNET_OK;
}

int pc_factor_stars(spnet_pc_s* pc) {
  cudaStream_t s = pc->op->stream;
  if (pc->S == 0) return SPNET_OK;
  if (pc->sum_s > INT32_MAX)
    return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: the stars hold more than 2^31-1 entries in total");
  if (pc->max_star > STREAM_MAX_N)
    return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: a star holds more than " +
                                           std::to_string(STREAM_MAX_N) + " dofs");
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const int nmax = pc->max_star;
  if (nmax > 65535) return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: a star beyond 65535 dofs");
  int max_row = 0;
  {
    int* d = nullptr;
    SPNET_TRY(tmp.get(&d, 1));
    SPNET_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(int), s));
    note_launch();
    k_max_row<<<4 * num_sms(), 256, 0, s>>>(pc->N, pc->K.ptr, d);
    SPNET_CUDA_TRY(cudaGetLastError());
    SPNET_CUDA_TRY(cudaMemcpyAsync(&max_row, d, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  }
  const int acap = adjacency_cap(max_row - 1);
  const int64_t hot = hot_bytes(nmax, acap);
  // hot arrays in shared memory when four warps' worth fit in 200 KiB, one
  // block of four warps per SM at least; otherwise everything in global scratch
  const int hot_in_smem = 4 * hot <= 200 * 1024 ? 1 : 0;
  int wpb_blocks = hot_in_smem ? (int)((200 * 1024) / (4 * hot)) : 4;  // blocks per SM
  if (wpb_blocks < 1) wpb_blocks = 1;
  if (wpb_blocks > 4) wpb_blocks = 4;
  if (hot_in_smem) {
    static std::atomic<bool> attr_set[64];  // per device
    int dev = 0;
    SPNET_CUDA_TRY(cudaGetDevice(&dev));
    dev &= 63;
    if (!attr_set[dev]) {
      SPNET_CUDA_TRY(cudaFuncSetAttribute(k_star_symbolic, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr_set[dev] = true;
    }
  }
  // per-warp scratch for a dense block of core_max nodes; warps within a 1 GiB budget
  // (stars beyond 4 CORE_FIRST dofs start at four times the capacity: their
  // eliminations end in larger blocks and a failed first pass costs a launch)
  int core_max = nmax <= 4 * CORE_FIRST ? (nmax < CORE_FIRST ? nmax : CORE_FIRST) : 4 * CORE_FIRST;
  int64_t stride = 0, warps = 0;
  char* scratch = nullptr;
  auto size_scratch = [&]() -> int {
    stride = cold_bytes(nmax, core_max, acap) + (hot_in_smem ? 0 : align_up(hot, 256));
    warps = (int64_t)4 * wpb_blocks * num_sms();
    const int64_t budget = (int64_t)1 << 30;
    if (warps * stride > budget) warps = budget / stride;
    if (warps < 4) warps = 4;
    if (warps > pc->S) warps = pc->S;
    warps = (warps + 3) / 4 * 4;
    if (scratch) tmp.release(scratch);
    scratch = nullptr;
    return tmp.get(&scratch, warps * stride);
  };
  SPNET_TRY(size_scratch());
  int* counters = nullptr;  // [0] next star, [2..3] pool top (u64)
  SPNET_TRY(tmp.get(&counters, 4));
  SPNET_TRY(pc->mem.get(&pc->star_off, pc->S));
  SPNET_TRY(pc->mem.get(&pc->star_lev, pc->S));
  SPNET_TRY(pc->mem.get(&pc->star_nnz, pc->S));
  SPNET_TRY(pc->mem.get(&pc->star_core, pc->S));
  // pool estimate: per dof 28 bytes + ~4 factor entries of 32 bytes, per star 64
  int64_t cap = pc->sum_s * (28 + 4 * 32) + (int64_t)pc->S * 64 + (1 << 20);
  int* flags = pc->op->dflags;
  for (int attempt = 0; attempt < 8; ++attempt) {
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
    A.core_max = core_max;
    A.pool = pc->pool;
    A.pool_cap = cap;
    A.pool_top = (unsigned long long*)(counters + 2);
    A.star_off = pc->star_off;
    A.star_lev = pc->star_lev;
    A.star_nnz = pc->star_nnz;
    A.star_core = pc->star_core;
    A.flags = flags;
    A.next = counters;
    A.vbytes = 8;  // the set-up blobs keep FP64 values; the solve sections are packed later
    A.cap = acap;
    A.patch = pc->star_rule;
    A.q1w = pc->patch_w;
    A.N = pc->N;
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
    if ((h & FLAG_STAR_BIG) && !(h & ~(FLAG_STAR_BIG | FLAG_POOL)) && core_max < nmax) {
      // a dense block beyond the scratch: again with four times the capacity
      core_max = core_max * 4 < nmax ? core_max * 4 : nmax;
      SPNET_TRY(size_scratch());
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
  note_launch();
  ProfScope ps(KID_STAR_NUMERIC, s);
  // a warp per star, or a block per star when some star exceeds 1024 dofs
  if (pc->max_star > 1024)
    k_star_numeric<NT><<<pc->S, NT, 0, s>>>(pc->S, pc->pool, pc->star_off, pc->K.ptr, pc->K.col, pc->K.val, 8,
                                            flags);
  else
    k_star_numeric<32><<<(pc->S + NT / 32 - 1) / (NT / 32), NT, 0, s>>>(pc->S, pc->pool, pc->star_off, pc->K.ptr,
                                                                        pc->K.col, pc->K.val, 8, flags);
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
  // the solve streams (and the panel solves of dense blocks for FP32 blocks of right-hand
  // sides); the set-up blobs are released
  SPNET_TRY(pack_streams(pc, tmp, lev, nz));
  if (pc->precision == SPNET_PREC_MIXED && pc->batch_rhs >= 2 && pc->panels) SPNET_TRY(pack_panels(pc, tmp));
  pc->mem.release(pc->pool);
  pc->pool = nullptr;
  return SPNET_OK;
}

}  // namespace spnet
