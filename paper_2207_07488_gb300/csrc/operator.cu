// The free-dof operator A = K_II and the lifting block K_ID (Section 3), and
// the CSR SpMV used by the PCG iteration.
#include <cmath>

#include "spnet_internal.cuh"

namespace spnet {

__global__ void k_check_csr(int64_t n, const int64_t* ptr, const int32_t* col, const double* val,
                            int* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = ptr[i], b = ptr[i + 1];
    if (b < a) {
      atomicOr(flags, FLAG_BAD_INPUT);
      continue;
    }
    int32_t prev = -1;
    for (int64_t k = a; k < b; ++k) {
      int32_t c = col[k];
      if (c < 0 || c >= n) atomicOr(flags, FLAG_BAD_INPUT);
      if (c <= prev) atomicOr(flags, FLAG_UNSORTED);
      if (!isfinite(val[k])) atomicOr(flags, FLAG_NONFINITE);
      prev = c;
    }
  }
}

__global__ void k_check_coords(int64_t n, int dim, const double* X, double l0, double l1, double l2,
                               int* flags) {
  double l[3] = {l0, l1, l2};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int a = 0; a < dim; ++a) {
      double x = X[i * dim + a];
      if (!(x >= 0.0 && x <= l[a])) atomicOr(flags, FLAG_OUT_OF_BOX);
    }
}

__global__ void k_mark_dirichlet(int64_t nd, const int64_t* dd, int64_t n_dof, int64_t* free_of,
                                 int32_t* is_free, int* flags) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nd;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = dd[k];
    if (v < 0 || v >= n_dof || (k > 0 && dd[k - 1] >= v)) {
      atomicOr(flags, FLAG_BAD_INPUT);
      continue;
    }
    is_free[v] = 0;
    free_of[v] = -(k + 2);  // -(position in the Dirichlet list) - 2
  }
}

__global__ void k_free_index(int64_t n_dof, const int32_t* is_free, const int64_t* pos,
                             int64_t* free_of, int64_t* free_dofs) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_dof;
       v += (int64_t)gridDim.x * blockDim.x)
    if (is_free[v]) {
      free_of[v] = pos[v];
      free_dofs[pos[v]] = v;
    }
}

// row lengths of K_II and K_ID
__global__ void k_split_count(int64_t n_free, const int64_t* free_dofs, const int64_t* free_of,
                              const int64_t* ptr, const int32_t* col, int32_t* len_ff,
                              int32_t* len_fd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_free;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = free_dofs[i];
    int32_t a = 0, b = 0;
    for (int64_t k = ptr[v]; k < ptr[v + 1]; ++k) {
      if (free_of[col[k]] >= 0) ++a; else ++b;
    }
    len_ff[i] = a;
    len_fd[i] = b;
  }
}

__global__ void k_split_fill(int64_t n_free, const int64_t* free_dofs, const int64_t* free_of,
                             const int64_t* ptr, const int32_t* col, const double* val,
                             const int64_t* pff, int32_t* cff, double* vff, const int64_t* pfd,
                             int32_t* cfd, double* vfd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_free;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = free_dofs[i];
    int64_t a = pff[i], b = pfd[i];
    for (int64_t k = ptr[v]; k < ptr[v + 1]; ++k) {
      int64_t f = free_of[col[k]];
      if (f >= 0) {
        cff[a] = (int32_t)f;
        vff[a++] = val[k];
      } else {
        cfd[b] = (int32_t)(-f - 2);
        vfd[b++] = val[k];
      }
    }
  }
}

// symmetry of A and positive diagonal
__global__ void k_check_sym(int64_t n, const int64_t* ptr, const int32_t* col, const double* val,
                            int* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bool has_diag = false;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      int32_t j = col[k];
      double v = val[k];
      if (j == i) {
        has_diag = true;
        if (!(v > 0.0)) atomicOr(flags, FLAG_NOT_SPD);
        continue;
      }
      // binary search (i) in row j
      int64_t lo = ptr[j], hi = ptr[j + 1] - 1;
      double vt = 0.0;
      bool found = false;
      while (lo <= hi) {
        int64_t m = (lo + hi) >> 1;
        int32_t c = col[m];
        if (c == i) {
          vt = val[m];
          found = true;
          break;
        }
        if (c < i) lo = m + 1; else hi = m - 1;
      }
      double tol = 1e-12 * fmax(fabs(v), fabs(vt));
      if (!found && v != 0.0) atomicOr(flags, FLAG_ASYM);
      if (found && fabs(v - vt) > tol) atomicOr(flags, FLAG_ASYM);
    }
    if (!has_diag) atomicOr(flags, FLAG_NOT_SPD);
  }
}

// ---------------------------------------------------------------------------
// SpMV y = A x with a fused partial dot (x, y): L lanes per row.
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(256) k_spmv(int64_t n, const int64_t* __restrict__ ptr,
                                              const int32_t* __restrict__ col,
                                              const double* __restrict__ val,
                                              const double* __restrict__ x, double* __restrict__ y,
                                              double* partial, const int* done) {
  if (done && *done) return;
  __shared__ double sh[256 / 32];
  constexpr int RPW = 32 / L;  // rows per warp pass
  const int lane = threadIdx.x & 31;
  const int sub = lane % L;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  // the loop bound is uniform across the warp, so every lane reaches the shuffles
  for (int64_t base = gwarp * RPW; base < n; base += nwarps * RPW) {
    const int64_t row = base + lane / L;
    const bool valid = row < n;
    double s = 0.0;
    if (valid) {
      const int64_t a = ptr[row], b = ptr[row + 1];
      for (int64_t k = a + sub; k < b; k += L) s = fma(val[k], __ldg(&x[col[k]]), s);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, L);
    if (valid && sub == 0) {
      y[row] = s;
      if (partial) dot = fma(s, x[row], dot);
    }
  }
  if (!partial) return;
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0) sh[threadIdx.x >> 5] = dot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

void launch_spmv(const Csr& A, const double* x, double* y, double* partial, int G, int lanes,
                 const int* done, cudaStream_t s) {
  note_launch();
  ProfScope ps(KID_SPMV, s);
  switch (lanes) {
    case 1: k_spmv<1><<<G, 256, 0, s>>>(A.n, A.ptr, A.col, A.val, x, y, partial, done); break;
    case 2: k_spmv<2><<<G, 256, 0, s>>>(A.n, A.ptr, A.col, A.val, x, y, partial, done); break;
    case 4: k_spmv<4><<<G, 256, 0, s>>>(A.n, A.ptr, A.col, A.val, x, y, partial, done); break;
    case 8: k_spmv<8><<<G, 256, 0, s>>>(A.n, A.ptr, A.col, A.val, x, y, partial, done); break;
    case 16: k_spmv<16><<<G, 256, 0, s>>>(A.n, A.ptr, A.col, A.val, x, y, partial, done); break;
    default: k_spmv<32><<<G, 256, 0, s>>>(A.n, A.ptr, A.col, A.val, x, y, partial, done); break;
  }
}

// lanes per row: one thread per row for the short rows of networks (a few
// entries), a few lanes per row as rows get longer
int choose_spmv_lanes(const Csr& A) {
  double avg = A.n > 0 ? (double)A.nnz / (double)A.n : 1.0;
  if (avg <= 6) return 1;
  if (avg <= 12) return 2;
  if (avg <= 24) return 4;
  if (avg <= 48) return 8;
  if (avg <= 96) return 16;
  return 32;
}

// everything after the handle exists; temporary buffers are released (on the
// operator's stream) before the caller decides whether to keep the handle
static int build_operator_fill(spnet_op_s* op, const double* coords, const int64_t* row_ptr,
                               const int32_t* col_idx, const double* vals, const int64_t* dir,
                               int mem) {
  const int dim = op->dim;
  const int64_t n_nodes = op->n_nodes, n_dir = op->n_dir;
  cudaStream_t s = op->stream;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const int64_t nd = op->n_dof;
  int64_t nnz = 0;
  int rc;
  if (mem == SPNET_MEM_HOST) {
    nnz = row_ptr[nd];
  } else {
    if (cudaMemcpyAsync(&nnz, row_ptr + nd, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return (fail(SPNET_ERR_CUDA, "build_network_operator: reading nnz"));
  }
  if (nnz < 0 || nnz >= ((int64_t)1 << 31)) return (fail(SPNET_ERR_UNSUPPORTED, "nnz out of range"));
  int64_t *d_ptr = nullptr;
  int32_t* d_col = nullptr;
  double* d_val = nullptr;
  if ((rc = tmp.get(&d_ptr, nd + 1)) || (rc = tmp.get(&d_col, nnz)) || (rc = tmp.get(&d_val, nnz)))
    return rc;
  if ((rc = copy_in(row_ptr, d_ptr, sizeof(int64_t) * (nd + 1), mem, s)) ||
      (rc = copy_in(col_idx, d_col, sizeof(int32_t) * nnz, mem, s)) ||
      (rc = copy_in(vals, d_val, sizeof(double) * nnz, mem, s)))
    return rc;
  if ((rc = op->mem.get(&op->coords, n_nodes * dim)) || (rc = op->mem.get(&op->dflags, 1)) ||
      (rc = op->mem.get(&op->dir_dofs, n_dir)) || (rc = op->mem.get(&op->free_of, nd)))
    return rc;
  if ((rc = copy_in(coords, op->coords, sizeof(double) * n_nodes * dim, mem, s)) ||
      (rc = copy_in(dir, op->dir_dofs, sizeof(int64_t) * n_dir, mem, s)))
    return rc;
  cudaMemsetAsync(op->dflags, 0, sizeof(int), s);
  int grid = 4 * num_sms();
  note_launch();
  k_check_csr<<<grid, 256, 0, s>>>(nd, d_ptr, d_col, d_val, op->dflags);
  note_launch();
  k_check_coords<<<grid, 256, 0, s>>>(n_nodes, dim, op->coords, op->domain[0], op->domain[1],
                                      op->domain[2], op->dflags);
  int32_t* is_free = nullptr;
  int64_t* pos = nullptr;
  if ((rc = tmp.get(&is_free, nd)) || (rc = tmp.get(&pos, nd + 1))) return rc;
  // every dof starts free; the Dirichlet ones are then cleared
  cudaMemsetAsync(op->free_of, 0xff, sizeof(int64_t) * nd, s);
  fill_i32(is_free, nd, 1, s);
  note_launch();
  k_mark_dirichlet<<<grid, 256, 0, s>>>(n_dir, op->dir_dofs, nd, op->free_of, is_free, op->dflags);
  if ((rc = check_flags(op->dflags, s, "build_network_operator"))) return rc;
  if ((rc = scan_exclusive(is_free, pos, nd, s, tmp))) return rc;
  int64_t n_free = 0;
  cudaMemcpyAsync(&n_free, pos + nd, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  op->n_free = n_free;
  if (n_free != nd - n_dir) return (fail(SPNET_ERR_BAD_INPUT, "duplicate Dirichlet dofs"));
  if ((rc = op->mem.get(&op->free_dofs, n_free))) return rc;
  note_launch();
  k_free_index<<<grid, 256, 0, s>>>(nd, is_free, pos, op->free_of, op->free_dofs);
  int32_t *len_ff = nullptr, *len_fd = nullptr;
  if ((rc = tmp.get(&len_ff, n_free + 1)) || (rc = tmp.get(&len_fd, n_free + 1))) return rc;
  note_launch();
  k_split_count<<<grid, 256, 0, s>>>(n_free, op->free_dofs, op->free_of, d_ptr, d_col, len_ff, len_fd);
  op->ff.n = op->fd.n = n_free;
  if ((rc = op->mem.get(&op->ff.ptr, n_free + 1)) || (rc = op->mem.get(&op->fd.ptr, n_free + 1)))
    return rc;
  if ((rc = scan_exclusive(len_ff, op->ff.ptr, n_free, s, tmp)) ||
      (rc = scan_exclusive(len_fd, op->fd.ptr, n_free, s, tmp)))
    return rc;
  cudaMemcpyAsync(&op->ff.nnz, op->ff.ptr + n_free, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&op->fd.nnz, op->fd.ptr + n_free, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if ((rc = op->mem.get(&op->ff.col, op->ff.nnz)) || (rc = op->mem.get(&op->ff.val, op->ff.nnz)) ||
      (rc = op->mem.get(&op->fd.col, op->fd.nnz)) || (rc = op->mem.get(&op->fd.val, op->fd.nnz)))
    return rc;
  note_launch();
  k_split_fill<<<grid, 256, 0, s>>>(n_free, op->free_dofs, op->free_of, d_ptr, d_col, d_val,
                                    op->ff.ptr, op->ff.col, op->ff.val, op->fd.ptr, op->fd.col,
                                    op->fd.val);
  note_launch();
  k_check_sym<<<grid, 256, 0, s>>>(n_free, op->ff.ptr, op->ff.col, op->ff.val, op->dflags);
  if ((rc = check_flags(op->dflags, s, "build_network_operator"))) return rc;
  if (cudaGetLastError() != cudaSuccess) return (fail(SPNET_ERR_CUDA, "build_network_operator: launch failed"));
  return SPNET_OK;
}

int build_operator(int dim, int ndof, int64_t n_nodes, const double* coords, const int64_t* row_ptr,
                   const int32_t* col_idx, const double* vals, int64_t n_dir, const int64_t* dir,
                   const double* domain_hi, int mem, cudaStream_t s, spnet_op_s** out) {
  if (dim < 2 || dim > 3) return fail(SPNET_ERR_BAD_INPUT, "build_network_operator: dim must be 2 or 3");
  if (ndof != 1 && ndof != 3) return fail(SPNET_ERR_BAD_INPUT, "build_network_operator: ndof must be 1 or 3");
  if (n_nodes <= 0 || n_dir < 0) return fail(SPNET_ERR_BAD_INPUT, "build_network_operator: bad sizes");
  if (n_nodes * ndof >= ((int64_t)1 << 31))
    return fail(SPNET_ERR_UNSUPPORTED, "build_network_operator: more than 2^31 dofs");
  for (int a = 0; a < dim; ++a)
    if (!(domain_hi[a] > 0.0)) return fail(SPNET_ERR_BAD_INPUT, "build_network_operator: domain side <= 0");
  int dev = 0;
  SPNET_CUDA_TRY(cudaGetDevice(&dev));
  spnet_op_s* op = new spnet_op_s();
  op->device = dev;
  if (s == 0) {
    // the legacy default stream cannot be captured into CUDA graphs: work on a
    // private stream instead (every call synchronises it before returning)
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      delete op;
      return fail(SPNET_ERR_CUDA, "build_network_operator: cannot create a stream");
    }
    op->own_stream = true;
  }
  op->dim = dim;
  op->ndof = ndof;
  op->n_nodes = n_nodes;
  op->n_dof = n_nodes * ndof;
  op->n_dir = n_dir;
  op->stream = s;
  op->mem.stream = s;
  for (int a = 0; a < dim; ++a) op->domain[a] = domain_hi[a];
  const int rc = build_operator_fill(op, coords, row_ptr, col_idx, vals, dir, mem);
  if (rc != SPNET_OK) {
    op->mem.free_all();
    cudaStreamSynchronize(s);
    if (op->own_stream) cudaStreamDestroy(s);
    delete op;
    return rc;
  }
  *out = op;
  return SPNET_OK;
}

}  // namespace spnet
