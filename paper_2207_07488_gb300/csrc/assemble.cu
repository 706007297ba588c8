// Assembly of K from an edge list (Example 3.2 eq. scalarmodel; eq. tensile
// with the lateral term 0.1 c I of the 3-dof model).
//
// Every edge e = {i, j} adds c_e (d_i - d_j)(d_i - d_j)^T (scalar) or the 3x3
// block c_e (n n^T + 0.1 I) in the pattern [[+,-],[-,+]] (3 dofs per node).
// Node adjacency is gathered per node, sorted by (neighbour, edge id), and the
// CSR rows are written in that fixed order, so the result is deterministic.
#include <cmath>

#include "spnet_internal.cuh"

namespace spnet {

__global__ void k_edge_check(int64_t n_nodes, int64_t n_edges, const int64_t* edges,
                             const double* coef, const double* dirs, int model, int* deg,
                             int* flags) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_edges;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = edges[2 * e], j = edges[2 * e + 1];
    double c = coef[e];
    bool bad = i < 0 || j < 0 || i >= n_nodes || j >= n_nodes || i == j;
    bool nf = !isfinite(c);
    if (model == SPNET_MODEL_TRUSS3)
      for (int a = 0; a < 3; ++a) nf |= !isfinite(dirs[3 * e + a]);
    if (bad) atomicOr(flags, FLAG_BAD_INPUT);
    if (nf) atomicOr(flags, FLAG_NONFINITE);
    if (!bad) {
      atomicAdd(&deg[i], 1);
      atomicAdd(&deg[j], 1);
    }
  }
}

__global__ void k_edge_fill(int64_t n_nodes, int64_t n_edges, const int64_t* edges,
                            const int64_t* nptr, int* fill, int64_t* adj) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_edges;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = edges[2 * e], j = edges[2 * e + 1];
    if (i < 0 || j < 0 || i >= n_nodes || j >= n_nodes || i == j) continue;
    int si = atomicAdd(&fill[i], 1);
    int sj = atomicAdd(&fill[j], 1);
    // pack (neighbour, edge): neighbour in the high 32 bits so that sorting the
    // packed key sorts by neighbour first, then by edge id
    adj[nptr[i] + si] = (j << 32) | e;
    adj[nptr[j] + sj] = (i << 32) | e;
  }
}

// per node: sort its adjacency and count distinct neighbours -> rows of K
__global__ void k_node_sort(int64_t n_nodes, const int64_t* nptr, int64_t* adj, int ndof,
                            int32_t* rowlen) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_nodes;
       v += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = nptr[v], b = nptr[v + 1];
    for (int64_t k = a + 1; k < b; ++k) {  // insertion sort (degrees are small)
      int64_t key = adj[k];
      int64_t m = k - 1;
      while (m >= a && adj[m] > key) {
        adj[m + 1] = adj[m];
        --m;
      }
      adj[m + 1] = key;
    }
    int uniq = 0;
    int64_t prev = -1;
    for (int64_t k = a; k < b; ++k) {
      int64_t nb = adj[k] >> 32;
      if (nb != prev) ++uniq;
      prev = nb;
    }
    for (int c = 0; c < ndof; ++c) rowlen[v * ndof + c] = (uniq + 1) * ndof;
  }
}

__global__ void k_node_write(int64_t n_nodes, const int64_t* nptr, const int64_t* adj,
                             const double* coef, const double* dirs, int model,
                             const int64_t* row_ptr, int32_t* col, double* val) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_nodes;
       v += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = nptr[v], b = nptr[v + 1];
    if (model == SPNET_MODEL_SCALAR) {
      int64_t o = row_ptr[v];
      double diag = 0.0;
      bool diag_done = false;
      int64_t k = a;
      while (k < b) {
        int64_t nb = adj[k] >> 32;
        double s = 0.0;
        while (k < b && (adj[k] >> 32) == nb) {
          s += coef[adj[k] & 0xffffffffLL];
          ++k;
        }
        if (!diag_done && nb > v) {
          col[o] = (int32_t)v;
          o++;  // diagonal slot, value filled below
          diag_done = true;
        }
        col[o] = (int32_t)nb;
        val[o] = -s;
        diag += s;
        ++o;
      }
      // the diagonal is the sum of the off-diagonal magnitudes, in the same order
      if (!diag_done) {
        col[o] = (int32_t)v;
        val[o] = diag;
      } else {
        for (int64_t q = row_ptr[v]; q < row_ptr[v + 1]; ++q)
          if (col[q] == (int32_t)v) val[q] = diag;
      }
    } else {
      // three rows per node, each with 3*(uniq+1) entries: node blocks in
      // ascending neighbour order, the node's own block at its sorted place
      double D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      int64_t o0 = row_ptr[3 * v], o1 = row_ptr[3 * v + 1], o2 = row_ptr[3 * v + 2];
      int64_t slot = 0, dslot = -1;
      int64_t k = a;
      while (k < b) {
        int64_t nb = adj[k] >> 32;
        double Bk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        while (k < b && (adj[k] >> 32) == nb) {
          int64_t e = adj[k] & 0xffffffffLL;
          double c = coef[e];
          double n0 = dirs[3 * e], n1 = dirs[3 * e + 1], n2 = dirs[3 * e + 2];
          double nn[3] = {n0, n1, n2};
          for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) Bk[3 * r + s] += c * (nn[r] * nn[s] + (r == s ? 0.1 : 0.0));
          ++k;
        }
        if (dslot < 0 && nb > v) {
          dslot = slot;
          slot++;
        }
        for (int r = 0; r < 3; ++r) {
          int64_t orow = (r == 0 ? o0 : (r == 1 ? o1 : o2)) + 3 * slot;
          for (int s = 0; s < 3; ++s) {
            col[orow + s] = (int32_t)(3 * nb + s);
            val[orow + s] = -Bk[3 * r + s];
            D[3 * r + s] += Bk[3 * r + s];
          }
        }
        ++slot;
      }
      if (dslot < 0) dslot = slot;
      for (int r = 0; r < 3; ++r) {
        int64_t orow = (r == 0 ? o0 : (r == 1 ? o1 : o2)) + 3 * dslot;
        for (int s = 0; s < 3; ++s) {
          col[orow + s] = (int32_t)(3 * v + s);
          val[orow + s] = D[3 * r + s];
        }
      }
    }
  }
}

int assemble(int model, int64_t n_nodes, int64_t n_edges, const int64_t* edges,
             const double* coef, const double* dirs, int mem, cudaStream_t s, int64_t* row_ptr,
             int32_t* col, double* val, int64_t cap_nnz, int64_t* nnz_out) {
  if (model != SPNET_MODEL_SCALAR && model != SPNET_MODEL_TRUSS3)
    return fail(SPNET_ERR_BAD_INPUT, "spnet_assemble: unknown model");
  if (n_nodes <= 0 || n_edges < 0) return fail(SPNET_ERR_BAD_INPUT, "spnet_assemble: bad sizes");
  if (n_edges >= (int64_t)1 << 31 || n_nodes >= (int64_t)1 << 31)
    return fail(SPNET_ERR_UNSUPPORTED, "spnet_assemble: more than 2^31 nodes or edges");
  if (model == SPNET_MODEL_TRUSS3 && !dirs)
    return fail(SPNET_ERR_BAD_INPUT, "spnet_assemble: TRUSS3 needs dirs");
  const int ndof = model == SPNET_MODEL_SCALAR ? 1 : 3;
  const int64_t n_dof = n_nodes * ndof;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  int64_t *d_edges = nullptr, *nptr = nullptr, *adj = nullptr, *d_rowptr = nullptr;
  double *d_coef = nullptr, *d_dirs = nullptr;
  int *deg = nullptr, *flags = nullptr;
  int32_t* rowlen = nullptr;
  SPNET_TRY(tmp.get(&d_edges, 2 * n_edges));
  SPNET_TRY(tmp.get(&d_coef, n_edges));
  SPNET_TRY(copy_in(edges, d_edges, sizeof(int64_t) * 2 * n_edges, mem, s));
  SPNET_TRY(copy_in(coef, d_coef, sizeof(double) * n_edges, mem, s));
  if (model == SPNET_MODEL_TRUSS3) {
    SPNET_TRY(tmp.get(&d_dirs, 3 * n_edges));
    SPNET_TRY(copy_in(dirs, d_dirs, sizeof(double) * 3 * n_edges, mem, s));
  }
  SPNET_TRY(tmp.get(&deg, n_nodes + 1));
  SPNET_TRY(tmp.get(&flags, 1));
  SPNET_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int) * (n_nodes + 1), s));
  SPNET_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
  int grid = 4 * num_sms();
  note_launch();
  k_edge_check<<<grid, 256, 0, s>>>(n_nodes, n_edges, d_edges, d_coef, d_dirs, model, deg, flags);
  SPNET_TRY(check_flags(flags, s, "spnet_assemble"));
  SPNET_TRY(tmp.get(&nptr, n_nodes + 1));
  SPNET_TRY(scan_exclusive(deg, nptr, n_nodes, s, tmp));
  SPNET_TRY(tmp.get(&adj, 2 * n_edges));
  SPNET_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int) * (n_nodes + 1), s));
  note_launch();
  k_edge_fill<<<grid, 256, 0, s>>>(n_nodes, n_edges, d_edges, nptr, deg, adj);
  SPNET_TRY(tmp.get(&rowlen, n_dof + 1));
  note_launch();
  k_node_sort<<<grid, 128, 0, s>>>(n_nodes, nptr, adj, ndof, rowlen);
  if (mem == SPNET_MEM_DEVICE) {
    d_rowptr = row_ptr;
  } else {
    SPNET_TRY(tmp.get(&d_rowptr, n_dof + 1));
  }
  SPNET_TRY(scan_exclusive(rowlen, d_rowptr, n_dof, s, tmp));
  int64_t nnz = 0;
  SPNET_CUDA_TRY(cudaMemcpyAsync(&nnz, d_rowptr + n_dof, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  if (nnz > cap_nnz) return fail(SPNET_ERR_UNSUPPORTED, "spnet_assemble: cap_nnz too small");
  if (nnz >= ((int64_t)1 << 31)) return fail(SPNET_ERR_UNSUPPORTED, "spnet_assemble: nnz >= 2^31");
  int32_t* d_col = col;
  double* d_val = val;
  if (mem == SPNET_MEM_HOST) {
    SPNET_TRY(tmp.get(&d_col, nnz));
    SPNET_TRY(tmp.get(&d_val, nnz));
  }
  note_launch();
  k_node_write<<<grid, 128, 0, s>>>(n_nodes, nptr, adj, d_coef, d_dirs, model, d_rowptr, d_col, d_val);
  SPNET_CUDA_TRY(cudaGetLastError());
  if (mem == SPNET_MEM_HOST) {
    SPNET_TRY(copy_out(d_rowptr, row_ptr, sizeof(int64_t) * (n_dof + 1), mem, s));
    SPNET_TRY(copy_out(d_col, col, sizeof(int32_t) * nnz, mem, s));
    SPNET_TRY(copy_out(d_val, val, sizeof(double) * nnz, mem, s));
  }
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  if (nnz_out) *nnz_out = nnz;
  return SPNET_OK;
}

}  // namespace spnet

// ---------------------------------------------------------------------------
// The beam model (Example 3.3 with d = 2, n = 3; Section 6.3): eq. tensile without the
// lateral term, and eq. bend on node triples (x, y, z): for k = 1, 2 the triple adds
// E I / (L_y + L_z) (g_k . v)^2 with g_k = (eta_y / L_y on y, eta_z / L_z on z,
// -(eta_y / L_y + eta_z / L_z) on x); k = 2: eta_y = d_xy x e_3, eta_z = -d_xz x e_3 (the
// change of the angle between the two edges), k = 1: eta_y = eta_z = e_3.  Rows are
// built per node from its edges and the triples that hold it, in a fixed order.
// ---------------------------------------------------------------------------
namespace spnet {

constexpr int BEAM_ROW_MAX = 64;  // distinct nodes a node's rows may couple to

__global__ void k_triple_check(int64_t n_nodes, int64_t n_tri, const int64_t* tri, int* tcnt, int* flags) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tri; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = tri[4 * t], y = tri[4 * t + 1], z = tri[4 * t + 2];
    if (x < 0 || y < 0 || z < 0 || x >= n_nodes || y >= n_nodes || z >= n_nodes || x == y || x == z || y == z) {
      atomicOr(flags, FLAG_BAD_INPUT);
      continue;
    }
    atomicAdd(&tcnt[x], 1);
    atomicAdd(&tcnt[y], 1);
    atomicAdd(&tcnt[z], 1);
  }
}

__global__ void k_triple_fill(int64_t n_tri, const int64_t* tri, const int64_t* tptr, int* fill, int64_t* tlist) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tri; t += (int64_t)gridDim.x * blockDim.x) {
    for (int r = 0; r < 3; ++r) {
      const int64_t v = tri[4 * t + r];
      tlist[tptr[v] + atomicAdd(&fill[v], 1)] = (t << 2) | r;  // triple id, role of v
    }
  }
}

// sorted distinct nodes a node's rows couple to: itself, its edge neighbours, the members of its
// triples; returns the count, or -1 past BEAM_ROW_MAX
__device__ int beam_row_nodes(int64_t v, const int64_t* nptr, const int64_t* adj, const int64_t* tptr,
                              int64_t* tlist, const int64_t* tri, int64_t* out) {
  int cnt = 0;
  auto add = [&](int64_t u) {
    for (int i = 0; i < cnt; ++i)
      if (out[i] == u) return true;
    if (cnt == BEAM_ROW_MAX) return false;
    int i = cnt++;
    while (i > 0 && out[i - 1] > u) {  // keep ascending
      out[i] = out[i - 1];
      --i;
    }
    out[i] = u;
    return true;
  };
  bool ok = add(v);
  for (int64_t k = nptr[v]; k < nptr[v + 1]; ++k) ok = ok && add(adj[k] >> 32);
  for (int64_t k = tptr[v]; k < tptr[v + 1]; ++k) {
    const int64_t t = tlist[k] >> 2;
    for (int r = 0; r < 3; ++r) ok = ok && add(tri[4 * t + r]);
  }
  return ok ? cnt : -1;
}

__global__ void k_beam_rowlen(int64_t n_nodes, const int64_t* nptr, const int64_t* adj, const int64_t* tptr,
                              int64_t* tlist, const int64_t* tri, int32_t* rowlen, int* flags) {
  int64_t nodes[BEAM_ROW_MAX];
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_nodes; v += (int64_t)gridDim.x * blockDim.x) {
    // the node's triples in ascending (triple, role) order: a fixed order of the sums
    for (int64_t k = tptr[v] + 1; k < tptr[v + 1]; ++k) {
      const int64_t key = tlist[k];
      int64_t m = k - 1;
      while (m >= tptr[v] && tlist[m] > key) {
        tlist[m + 1] = tlist[m];
        --m;
      }
      tlist[m + 1] = key;
    }
    const int c = beam_row_nodes(v, nptr, adj, tptr, tlist, tri, nodes);
    if (c < 0) {
      atomicOr(flags, FLAG_STAR_BIG);
      for (int a = 0; a < 3; ++a) rowlen[3 * v + a] = 0;
      continue;
    }
    for (int a = 0; a < 3; ++a) rowlen[3 * v + a] = 3 * c;
  }
}

// the vector g_k of a triple, for the node in role r: 3 components
__device__ inline void beam_g(const double* X, const int64_t* tri, int64_t t, int k, int r, double* g) {
  const int64_t x = tri[4 * t], y = tri[4 * t + 1], z = tri[4 * t + 2];
  const double dyx = X[2 * y] - X[2 * x], dyy = X[2 * y + 1] - X[2 * x + 1];
  const double dzx = X[2 * z] - X[2 * x], dzy = X[2 * z + 1] - X[2 * x + 1];
  const double Ly = sqrt(dyx * dyx + dyy * dyy), Lz = sqrt(dzx * dzx + dzy * dzy);
  double ey[3], ez[3];
  if (k == 2) {  // d_xy x e_3 and -d_xz x e_3
    ey[0] = dyy / Ly; ey[1] = -dyx / Ly; ey[2] = 0.0;
    ez[0] = -dzy / Lz; ez[1] = dzx / Lz; ez[2] = 0.0;
  } else {
    ey[0] = ey[1] = ez[0] = ez[1] = 0.0;
    ey[2] = ez[2] = 1.0;
  }
  for (int a = 0; a < 3; ++a)
    g[a] = r == 1 ? ey[a] / Ly : r == 2 ? ez[a] / Lz : -(ey[a] / Ly + ez[a] / Lz);
}

__global__ void k_beam_write(int64_t n_nodes, const int64_t* nptr, const int64_t* adj, const int64_t* tptr,
                             const int64_t* tlist, const int64_t* tri, const double* X, const double* coef,
                             double EI, const int64_t* row_ptr, int32_t* col, double* val) {
  int64_t nodes[BEAM_ROW_MAX];
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_nodes; v += (int64_t)gridDim.x * blockDim.x) {
    const int c = beam_row_nodes(v, nptr, adj, tptr, (int64_t*)tlist, tri, nodes);
    if (c < 0) continue;
    for (int slot = 0; slot < c; ++slot) {
      const int64_t m = nodes[slot];
      double B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      // tensile: each edge v-u adds (gamma / L) d d^T to the (v, v) block and subtracts it from (v, u)
      for (int64_t k = nptr[v]; k < nptr[v + 1]; ++k) {
        const int64_t u = adj[k] >> 32, e = adj[k] & 0xffffffffLL;
        if (m != v && m != u) continue;
        const double dx = X[2 * u] - X[2 * v], dy = X[2 * u + 1] - X[2 * v + 1];
        const double L = sqrt(dx * dx + dy * dy);
        const double d[3] = {dx / L, dy / L, 0.0};
        const double w = (m == v ? 1.0 : -1.0) * coef[e] / L;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) B[3 * a + b] += w * (d[a] * d[b]);
      }
      // bending: each triple holding v and m adds E I / (L_y + L_z) g_k[v] g_k[m]^T, k = 1, 2.
      // Rows v and m sum the same terms in the same order (triples ascending, k = 2, 1)
      // and every product is formed as coefficient * (g[a] g[b]), so K is exactly symmetric.
      for (int64_t k = tptr[v]; k < tptr[v + 1]; ++k) {
        const int64_t t = tlist[k] >> 2;
        const int rv = (int)(tlist[k] & 3);
        for (int rm = 0; rm < 3; ++rm) {
          if (tri[4 * t + rm] != m) continue;
          const int64_t x = tri[4 * t], y = tri[4 * t + 1], z = tri[4 * t + 2];
          const double Ly = hypot(X[2 * y] - X[2 * x], X[2 * y + 1] - X[2 * x + 1]);
          const double Lz = hypot(X[2 * z] - X[2 * x], X[2 * z + 1] - X[2 * x + 1]);
          const double cb = EI / (Ly + Lz);
          for (int kk = 2; kk >= 1; --kk) {
            double gv[3], gm[3];
            beam_g(X, tri, t, kk, rv, gv);
            beam_g(X, tri, t, kk, rm, gm);
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) B[3 * a + b] += cb * (gv[a] * gm[b]);
          }
        }
      }
      for (int a = 0; a < 3; ++a) {
        const int64_t o = row_ptr[3 * v + a] + 3 * slot;
        for (int b = 0; b < 3; ++b) {
          col[o + b] = (int32_t)(3 * m + b);
          val[o + b] = B[3 * a + b];
        }
      }
    }
  }
}

int assemble_beam(int64_t n_nodes, int64_t n_edges, const int64_t* edges, const double* coords,
                  const double* coef, int64_t n_tri, const int64_t* tri, double EI, int mem, cudaStream_t s,
                  int64_t* row_ptr, int32_t* col, double* val, int64_t cap_nnz, int64_t* nnz_out) {
  if (n_nodes <= 0 || n_edges < 0 || n_tri < 0 || !(EI >= 0.0) || !std::isfinite(EI))
    return fail(SPNET_ERR_BAD_INPUT, "spnet_assemble_beam: bad sizes or E I");
  if (n_edges >= (int64_t)1 << 31 || 3 * n_nodes >= (int64_t)1 << 31)
    return fail(SPNET_ERR_UNSUPPORTED, "spnet_assemble_beam: more than 2^31 dofs or edges");
  const int64_t n_dof = 3 * n_nodes;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  int64_t *d_edges = nullptr, *d_tri = nullptr, *nptr = nullptr, *adj = nullptr, *tptr = nullptr, *tlist = nullptr,
          *d_rowptr = nullptr;
  double *d_coef = nullptr, *d_X = nullptr;
  int *deg = nullptr, *tcnt = nullptr, *flags = nullptr;
  int32_t* rowlen = nullptr;
  SPNET_TRY(tmp.get(&d_edges, 2 * n_edges + 1));
  SPNET_TRY(tmp.get(&d_coef, n_edges + 1));
  SPNET_TRY(tmp.get(&d_X, 2 * n_nodes));
  SPNET_TRY(tmp.get(&d_tri, 4 * n_tri + 1));
  SPNET_TRY(copy_in(edges, d_edges, sizeof(int64_t) * 2 * n_edges, mem, s));
  SPNET_TRY(copy_in(coef, d_coef, sizeof(double) * n_edges, mem, s));
  SPNET_TRY(copy_in(coords, d_X, sizeof(double) * 2 * n_nodes, mem, s));
  SPNET_TRY(copy_in(tri, d_tri, sizeof(int64_t) * 4 * n_tri, mem, s));
  SPNET_TRY(tmp.get(&deg, n_nodes + 1));
  SPNET_TRY(tmp.get(&tcnt, n_nodes + 1));
  SPNET_TRY(tmp.get(&flags, 1));
  SPNET_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int) * (n_nodes + 1), s));
  SPNET_CUDA_TRY(cudaMemsetAsync(tcnt, 0, sizeof(int) * (n_nodes + 1), s));
  SPNET_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
  const int grid = 4 * num_sms();
  note_launch();
  k_edge_check<<<grid, 256, 0, s>>>(n_nodes, n_edges, d_edges, d_coef, nullptr, SPNET_MODEL_SCALAR, deg, flags);
  note_launch();
  k_triple_check<<<grid, 256, 0, s>>>(n_nodes, n_tri, d_tri, tcnt, flags);
  SPNET_TRY(check_flags(flags, s, "spnet_assemble_beam"));
  SPNET_TRY(tmp.get(&nptr, n_nodes + 1));
  SPNET_TRY(scan_exclusive(deg, nptr, n_nodes, s, tmp));
  SPNET_TRY(tmp.get(&tptr, n_nodes + 1));
  SPNET_TRY(scan_exclusive(tcnt, tptr, n_nodes, s, tmp));
  SPNET_TRY(tmp.get(&adj, 2 * n_edges + 1));
  SPNET_TRY(tmp.get(&tlist, 3 * n_tri + 1));
  SPNET_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int) * (n_nodes + 1), s));
  SPNET_CUDA_TRY(cudaMemsetAsync(tcnt, 0, sizeof(int) * (n_nodes + 1), s));
  note_launch();
  k_edge_fill<<<grid, 256, 0, s>>>(n_nodes, n_edges, d_edges, nptr, deg, adj);
  note_launch();
  k_triple_fill<<<grid, 256, 0, s>>>(n_tri, d_tri, tptr, tcnt, tlist);
  SPNET_TRY(tmp.get(&rowlen, n_dof + 1));
  note_launch();
  k_node_sort<<<grid, 128, 0, s>>>(n_nodes, nptr, adj, 3, rowlen);  // sorts the edge lists
  note_launch();
  k_beam_rowlen<<<grid, 128, 0, s>>>(n_nodes, nptr, adj, tptr, tlist, d_tri, rowlen, flags);
  {
    int h = 0;
    SPNET_CUDA_TRY(cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPNET_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return fail(SPNET_ERR_UNSUPPORTED, "spnet_assemble_beam: a node couples to more than 64 nodes");
  }
  if (mem == SPNET_MEM_DEVICE) {
    d_rowptr = row_ptr;
  } else {
    SPNET_TRY(tmp.get(&d_rowptr, n_dof + 1));
  }
  SPNET_TRY(scan_exclusive(rowlen, d_rowptr, n_dof, s, tmp));
  int64_t nnz = 0;
  SPNET_CUDA_TRY(cudaMemcpyAsync(&nnz, d_rowptr + n_dof, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  if (nnz > cap_nnz) return fail(SPNET_ERR_UNSUPPORTED, "spnet_assemble_beam: cap_nnz too small");
  if (nnz >= ((int64_t)1 << 31)) return fail(SPNET_ERR_UNSUPPORTED, "spnet_assemble_beam: nnz >= 2^31");
  int32_t* d_col = col;
  double* d_val = val;
  if (mem == SPNET_MEM_HOST) {
    SPNET_TRY(tmp.get(&d_col, nnz + 1));
    SPNET_TRY(tmp.get(&d_val, nnz + 1));
  }
  note_launch();
  k_beam_write<<<grid, 128, 0, s>>>(n_nodes, nptr, adj, tptr, tlist, d_tri, d_X, d_coef, EI, d_rowptr, d_col, d_val);
  SPNET_CUDA_TRY(cudaGetLastError());
  if (mem == SPNET_MEM_HOST) {
    SPNET_TRY(copy_out(d_rowptr, row_ptr, sizeof(int64_t) * (n_dof + 1), mem, s));
    SPNET_TRY(copy_out(d_col, col, sizeof(int32_t) * nnz, mem, s));
    SPNET_TRY(copy_out(d_val, val, sizeof(double) * nnz, mem, s));
  }
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  if (nnz_out) *nnz_out = nnz;
  return SPNET_OK;
}

}  // namespace spnet
