// Assembly of K from an edge list (Example 3.2 eq. scalarmodel; eq. tensile
// with the lateral term 0.1 c I of the 3-dof model).
//
// Every edge e = {i, j} adds c_e (d_i - d_j)(d_i - d_j)^T (scalar) or the 3x3
// block c_e (n n^T + 0.1 I) in the pattern [[+,-],[-,+]] (3 dofs per node).
// Node adjacency is gathered per node, sorted by (neighbour, edge id), and the
// CSR rows are written in that fixed order, so the result is deterministic.
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
