// Set-up of the preconditioner's structure (Sections 2.3 and 4.1):
//  - host element of every free dof by the half-open box rule and its Q1
//    values at the element's 2^d corners;
//  - the element-major renumbering of the free dofs ("pc order"), in which the
//    dofs of one element are contiguous, so that a star (the patch of the
//    2^d elements around a mesh node) is a union of 2^d contiguous ranges;
//  - A permuted into pc order;
//  - the coarse dofs (mesh node, component) and the stars;
//  - the Galerkin matrix A_0 = R_0 A R_0^T.
#include <cmath>

#include "spnet_internal.cuh"

namespace spnet {

// host element and local coordinates of a point; the arithmetic x * n / l, floor
// (Q1: the half-open rule) or ceil - 1 (P1: the lowest box whose closure holds the
// point, Remark 2.1), clamp, xi = x * n / l - e fixes the rounding of every weight.
__device__ __forceinline__ int host_element(const Mesh& m, const double* x, const double* l,
                                            double* xi) {
  int e = 0, stride = 1;
  for (int a = 0; a < m.d; ++a) {
    double s = x[a] * (double)m.n[a] / l[a];
    int ea = m.simplex ? (int)ceil(s) - 1 : (int)floor(s);
    if (ea > m.n[a] - 1) ea = m.n[a] - 1;
    if (ea < 0) ea = 0;
    xi[a] = s - (double)ea;
    e += ea * stride;
    stride *= m.n[a];
  }
  return e;
}

__global__ void k_elements(int64_t n_free, const int64_t* free_dofs, int ndof, const double* coords,
                           Mesh m, double l0, double l1, double l2, int32_t* elem_free,
                           int8_t* comp_free, int32_t* cnt) {
  double l[3] = {l0, l1, l2};
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n_free;
       f += (int64_t)gridDim.x * blockDim.x) {
    int64_t dof = free_dofs[f];
    int64_t node = dof / ndof;
    double x[3], xi[3];
    for (int a = 0; a < m.d; ++a) x[a] = coords[node * m.d + a];
    int e = host_element(m, x, l, xi);
    elem_free[f] = e;
    comp_free[f] = (int8_t)(dof % ndof);
    atomicAdd(&cnt[e], 1);
  }
}

__global__ void k_place(int64_t n_free, const int32_t* elem_free, const int64_t* eptr, int32_t* fill,
                        int32_t* tmp) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n_free;
       f += (int64_t)gridDim.x * blockDim.x) {
    int e = elem_free[f];
    int s = atomicAdd(&fill[e], 1);
    tmp[eptr[e] + s] = (int32_t)f;
  }
}

// sort each element's free indices ascending (rank of each key in its segment)
__global__ void k_segment_sort(int n_elem, const int64_t* eptr, const int32_t* tmp, int32_t* perm) {
  for (int e = blockIdx.x; e < n_elem; e += gridDim.x) {
    int64_t a = eptr[e], b = eptr[e + 1];
    for (int64_t t = a + threadIdx.x; t < b; t += blockDim.x) {
      int32_t key = tmp[t];
      int64_t rank = 0;
      for (int64_t u = a; u < b; ++u) rank += tmp[u] < key;
      perm[a + rank] = key;
    }
  }
}

__global__ void k_pc_maps(int64_t N, const int32_t* perm, const int32_t* elem_free,
                          const int8_t* comp_free, const int64_t* free_dofs, int ndof,
                          const double* coords, Mesh m, double l0, double l1, double l2,
                          int32_t* iperm, int32_t* elem_of, int8_t* comp_of, double* q1w, double* xio,
                          float* xio32, double* vind) {
  double l[3] = {l0, l1, l2};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    int32_t f = perm[p];
    iperm[f] = (int32_t)p;
    elem_of[p] = elem_free[f];
    comp_of[p] = comp_free[f];
    int64_t node = free_dofs[f] / ndof;
    double x[3], xi[3];
    for (int a = 0; a < m.d; ++a) x[a] = coords[node * m.d + a];
    host_element(m, x, l, xi);
    for (int a = 0; a < m.d; ++a) {
      xio[(int64_t)a * N + p] = xi[a];
      xio32[(int64_t)a * N + p] = (float)xi[a];
    }
    if (m.simplex) {  // P1 on the Kuhn simplex; vind: 1 at the corners that are its vertices
      const double t3[3] = {xi[0], xi[1], m.d == 3 ? xi[2] : 0.0};
      double w[8];
      int vm;
      if (m.nc == 4) {
        double w4[4];
        p1_from_xi<4>(t3, w4);
        for (int c = 0; c < 4; ++c) w[c] = w4[c];
        vm = p1_vertex_mask<4>(t3);
      } else {
        p1_from_xi<8>(t3, w);
        vm = p1_vertex_mask<8>(t3);
      }
      for (int c = 0; c < m.nc; ++c) {
        q1w[(int64_t)c * N + p] = w[c];
        if (vind) vind[(int64_t)c * N + p] = (vm >> c) & 1 ? 1.0 : 0.0;
      }
    } else {
      for (int c = 0; c < m.nc; ++c) {
        double w = 1.0;
        for (int a = 0; a < m.d; ++a) w *= ((c >> a) & 1) ? xi[a] : (1.0 - xi[a]);
        q1w[(int64_t)c * N + p] = w;
      }
    }
  }
}

__global__ void k_perm_rowlen(int64_t N, const int32_t* perm, const int64_t* fptr, int32_t* len) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    int32_t f = perm[p];
    len[p] = (int32_t)(fptr[f + 1] - fptr[f]);
  }
}

__global__ void k_perm_fill(int64_t N, const int32_t* perm, const int32_t* iperm, const int64_t* fptr,
                            const int32_t* fcol, const double* fval, const int64_t* kptr,
                            int32_t* kcol, double* kval) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    int32_t f = perm[p];
    int64_t a = kptr[p], len = kptr[p + 1] - a;
    int64_t src = fptr[f];
    for (int64_t t = 0; t < len; ++t) {  // insertion sort by new column
      int32_t c = iperm[fcol[src + t]];
      double v = fval[src + t];
      int64_t q = a + t - 1;
      while (q >= a && kcol[q] > c) {
        kcol[q + 1] = kcol[q];
        kval[q + 1] = kval[q];
        --q;
      }
      kcol[q + 1] = c;
      kval[q + 1] = v;
    }
  }
}

// mark (mesh node, component) pairs whose basis function is nonzero at a free dof
__global__ void k_coarse_support(int64_t N, const int32_t* elem_of, const int8_t* comp_of,
                                 const double* q1w, Mesh m, int ndof, int32_t* flag) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    int e = elem_of[p];
    for (int c = 0; c < m.nc; ++c)
      if (q1w[(int64_t)c * N + p] != 0.0) flag[(int64_t)mesh_of(m, e, c) * ndof + comp_of[p]] = 1;
  }
}

__global__ void k_coarse_faces(int n_mesh, Mesh m, int ndof, int f0, int f1, int f2, int32_t* flag) {
  int faces[3] = {f0, f1, f2};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_mesh; k += gridDim.x * blockDim.x) {
    int km[3];
    mesh_multi(m, k, km);
    for (int c = 0; c < ndof; ++c) {
      bool on = false;
      for (int a = 0; a < m.d; ++a) {
        if (((faces[c] >> (2 * a)) & 1) && km[a] == 0) on = true;
        if (((faces[c] >> (2 * a + 1)) & 1) && km[a] == m.n[a]) on = true;
      }
      if (on) flag[(int64_t)k * ndof + c] = 0;
    }
  }
}

__global__ void k_coarse_index(int64_t n, const int32_t* flag, const int64_t* pos, int32_t* cidx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    cidx[i] = flag[i] ? (int32_t)pos[i] : -1;
}

// star of mesh node k: in the chosen set and with at least one free dof
__global__ void k_star_count(int n_mesh, Mesh m, int star_set, const int64_t* eptr, int32_t* sflag,
                             int32_t* scnt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_mesh; k += gridDim.x * blockDim.x) {
    int km[3];
    mesh_multi(m, k, km);
    bool in = true;
    if (star_set == SPNET_STARS_INTERIOR)
      for (int a = 0; a < m.d; ++a) in = in && km[a] > 0 && km[a] < m.n[a];
    int64_t cnt = 0;
    for (int cp = 0; cp < m.nc; ++cp) {
      int e = elem_around(m, km, cp);
      if (e >= 0) cnt += eptr[e + 1] - eptr[e];
    }
    sflag[k] = (in && cnt > 0) ? 1 : 0;
    scnt[k] = (in && cnt > 0) ? (int32_t)cnt : 0;
  }
}

// with a patch test in use (support patches, P1 element patches) a free dof may lie in no
// star: the star term is then zero there and B singular
__global__ void k_star_cover(int64_t N, Mesh m, const int32_t* elem_of, const double* patch_w,
                             const int32_t* star_of_mesh, int* flags) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int e = elem_of[p];
    bool cov = false;
    for (int c = 0; c < m.nc; ++c)
      cov |= star_of_mesh[mesh_of(m, e, c)] >= 0 && patch_w[(int64_t)c * N + p] != 0.0;
    if (!cov) atomicOr(flags, FLAG_UNCOVERED);
  }
}

__global__ void k_star_index(int n_mesh, const int32_t* sflag, const int64_t* spos,
                             const int32_t* scnt, int32_t* star_of_mesh, int32_t* star_mesh,
                             int32_t* star_n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_mesh; k += gridDim.x * blockDim.x) {
    if (sflag[k]) {
      int s = (int)spos[k];
      star_of_mesh[k] = s;
      star_mesh[s] = k;
      star_n[s] = scnt[k];
    } else {
      star_of_mesh[k] = -1;
    }
  }
}

// offset of element e inside the star at its corner c (stars list their
// elements e' = k - 1 + c' with c' ascending; e sits at c' = (nc-1) - c)
__global__ void k_elem_star_off(int n_elem, Mesh m, const int64_t* eptr, const int32_t* star_of_mesh,
                                int32_t* off) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_elem; e += gridDim.x * blockDim.x) {
    for (int c = 0; c < m.nc; ++c) {
      int k = mesh_of(m, e, c);
      int s = star_of_mesh[k];
      if (s < 0) {
        off[(int64_t)e * m.nc + c] = -1;
        continue;
      }
      int km[3];
      mesh_multi(m, k, km);
      int cpe = (m.nc - 1) - c;
      int64_t o = 0;
      for (int cp = 0; cp < cpe; ++cp) {
        int e2 = elem_around(m, km, cp);
        if (e2 >= 0) o += eptr[e2 + 1] - eptr[e2];
      }
      off[(int64_t)e * m.nc + c] = (int32_t)o;
    }
  }
}

__global__ void k_i64_to_i32(int64_t n, const int64_t* a, int32_t* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (int32_t)a[i];
}

int pc_setup_structure(spnet_pc_s* pc) {
  spnet_op_s* op = pc->op;
  cudaStream_t s = op->stream;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  const int64_t N = op->n_free;
  const Mesh m = mesh_of_pc(pc);
  const int grid = 4 * num_sms();
  pc->N = N;
  // host elements and counts
  int32_t *elem_free = nullptr, *cnt = nullptr, *fill = nullptr, *ptmp = nullptr;
  int8_t* comp_free = nullptr;
  int64_t* eptr = nullptr;
  SPNET_TRY(tmp.get(&elem_free, N));
  SPNET_TRY(tmp.get(&comp_free, N));
  SPNET_TRY(tmp.get(&cnt, pc->n_elem + 1));
  SPNET_TRY(tmp.get(&fill, pc->n_elem + 1));
  SPNET_TRY(tmp.get(&eptr, pc->n_elem + 1));
  SPNET_TRY(tmp.get(&ptmp, N));
  SPNET_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (pc->n_elem + 1), s));
  SPNET_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int32_t) * (pc->n_elem + 1), s));
  note_launch();
  k_elements<<<grid, 256, 0, s>>>(N, op->free_dofs, op->ndof, op->coords, m, op->domain[0],
                                  op->domain[1], op->domain[2], elem_free, comp_free, cnt);
  SPNET_TRY(scan_exclusive(cnt, eptr, pc->n_elem, s, tmp));
  note_launch();
  k_place<<<grid, 256, 0, s>>>(N, elem_free, eptr, fill, ptmp);
  SPNET_TRY(pc->mem.get(&pc->perm, N));
  SPNET_TRY(pc->mem.get(&pc->iperm, N));
  SPNET_TRY(pc->mem.get(&pc->elem_of, N));
  SPNET_TRY(pc->mem.get(&pc->comp_of, N));
  SPNET_TRY(pc->mem.get(&pc->elem_ptr, pc->n_elem + 1));
  SPNET_TRY(pc->mem.get(&pc->q1w, (int64_t)pc->nc * N));
  SPNET_TRY(pc->mem.get(&pc->xi, (int64_t)m.d * N));
  SPNET_TRY(pc->mem.get(&pc->xi32, (int64_t)m.d * N));
  // the star kernels' patch test (see spnet_pc_s::star_rule)
  double* vind = nullptr;
  if (pc->coarse_space == SPNET_COARSE_P1 && pc->patch == SPNET_PATCH_ELEMENT) {
    SPNET_TRY(pc->mem.get(&vind, (int64_t)pc->nc * N));
    pc->star_rule = SPNET_PATCH_SUPPORT;
    pc->patch_w = vind;
  } else {
    pc->star_rule = pc->patch;
    pc->patch_w = pc->q1w;
  }
  note_launch();
  k_segment_sort<<<grid, 128, 0, s>>>(pc->n_elem, eptr, ptmp, pc->perm);
  note_launch();
  k_i64_to_i32<<<grid, 256, 0, s>>>(pc->n_elem + 1, eptr, pc->elem_ptr);
  note_launch();
  k_pc_maps<<<grid, 256, 0, s>>>(N, pc->perm, elem_free, comp_free, op->free_dofs, op->ndof,
                                 op->coords, m, op->domain[0], op->domain[1], op->domain[2],
                                 pc->iperm, pc->elem_of, pc->comp_of, pc->q1w, pc->xi, pc->xi32, vind);
  // A in pc order
  int32_t* len = nullptr;
  SPNET_TRY(tmp.get(&len, N + 1));
  note_launch();
  k_perm_rowlen<<<grid, 256, 0, s>>>(N, pc->perm, op->ff.ptr, len);
  pc->K.n = N;
  pc->K.nnz = op->ff.nnz;
  SPNET_TRY(pc->mem.get(&pc->K.ptr, N + 1));
  SPNET_TRY(pc->mem.get(&pc->K.col, pc->K.nnz));
  SPNET_TRY(pc->mem.get(&pc->K.val, pc->K.nnz));
  SPNET_TRY(scan_exclusive(len, pc->K.ptr, N, s, tmp));
  note_launch();
  k_perm_fill<<<grid, 128, 0, s>>>(N, pc->perm, pc->iperm, op->ff.ptr, op->ff.col, op->ff.val,
                                   pc->K.ptr, pc->K.col, pc->K.val);
  // coarse dofs
  const int64_t nmc = (int64_t)pc->n_mesh * pc->ndof;
  int32_t* cflag = nullptr;
  int64_t* cpos = nullptr;
  SPNET_TRY(tmp.get(&cflag, nmc + 1));
  SPNET_TRY(tmp.get(&cpos, nmc + 1));
  SPNET_CUDA_TRY(cudaMemsetAsync(cflag, 0, sizeof(int32_t) * (nmc + 1), s));
  note_launch();
  k_coarse_support<<<grid, 256, 0, s>>>(N, pc->elem_of, pc->comp_of, pc->q1w, m, pc->ndof, cflag);
  int faces[3] = {0, 0, 0};
  for (int c = 0; c < pc->ndof; ++c) faces[c] = pc->gamma[c];
  note_launch();
  k_coarse_faces<<<grid, 256, 0, s>>>(pc->n_mesh, m, pc->ndof, faces[0], faces[1], faces[2], cflag);
  SPNET_TRY(scan_exclusive(cflag, cpos, nmc, s, tmp));
  SPNET_TRY(pc->mem.get(&pc->cidx, nmc));
  note_launch();
  k_coarse_index<<<grid, 256, 0, s>>>(nmc, cflag, cpos, pc->cidx);
  int64_t m0 = 0;
  SPNET_CUDA_TRY(cudaMemcpyAsync(&m0, cpos + nmc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  // stars
  int32_t *sflag = nullptr, *scnt = nullptr;
  int64_t* spos = nullptr;
  SPNET_TRY(tmp.get(&sflag, pc->n_mesh + 1));
  SPNET_TRY(tmp.get(&scnt, pc->n_mesh + 1));
  SPNET_TRY(tmp.get(&spos, pc->n_mesh + 1));
  note_launch();
  k_star_count<<<grid, 256, 0, s>>>(pc->n_mesh, m, pc->star_set, eptr, sflag, scnt);
  SPNET_TRY(scan_exclusive(sflag, spos, pc->n_mesh, s, tmp));
  int64_t S = 0;
  SPNET_CUDA_TRY(cudaMemcpyAsync(&S, spos + pc->n_mesh, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  pc->m0 = (int)m0;
  pc->S = (int)S;
  SPNET_TRY(pc->mem.get(&pc->star_of_mesh, pc->n_mesh));
  SPNET_TRY(pc->mem.get(&pc->star_mesh, S));
  SPNET_TRY(pc->mem.get(&pc->star_n, S));
  SPNET_TRY(pc->mem.get(&pc->star_ptr, S + 1));
  note_launch();
  k_star_index<<<grid, 256, 0, s>>>(pc->n_mesh, sflag, spos, scnt, pc->star_of_mesh, pc->star_mesh,
                                    pc->star_n);
  SPNET_TRY(scan_exclusive(pc->star_n, pc->star_ptr, S, s, tmp));
  SPNET_CUDA_TRY(cudaMemcpyAsync(&pc->sum_s, pc->star_ptr + S, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SPNET_TRY(pc->mem.get(&pc->elem_star_off, (int64_t)pc->n_elem * pc->nc));
  note_launch();
  k_elem_star_off<<<grid, 256, 0, s>>>(pc->n_elem, m, eptr, pc->star_of_mesh, pc->elem_star_off);
  if (S > 0 && pc->star_rule == SPNET_PATCH_SUPPORT) {
    SPNET_CUDA_TRY(cudaMemsetAsync(op->dflags, 0, sizeof(int), s));
    note_launch();
    k_star_cover<<<grid, 256, 0, s>>>(N, m, pc->elem_of, pc->patch_w, pc->star_of_mesh, op->dflags);
    SPNET_TRY(check_flags(op->dflags, s, "setup_preconditioner"));
  }
  // largest star
  std::vector<int32_t> sn(S);
  if (S > 0)
    SPNET_CUDA_TRY(cudaMemcpyAsync(sn.data(), pc->star_n, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  pc->max_star = 0;
  for (int32_t v : sn) pc->max_star = v > pc->max_star ? v : pc->max_star;
  SPNET_CUDA_TRY(cudaGetLastError());
  return SPNET_OK;
}

// A_0 = R_0 A R_0^T in two deterministic passes:
//   T = A R_0^T row by row (one thread per row of A: the row's entries times the
//       Q1 values of their columns, merged by coarse column in a fixed order),
//   A_0[k, :] = sum_{p in supp(phi_k)} phi_k(p) T[p, :] (one warp per coarse row,
//       the dofs of the support taken in order, lanes over the entries of T[p]).
constexpr int GAL_W = 512;

__global__ void k_galerkin_rowmax(int64_t N, const int64_t* kptr, int* mx) {
  int m = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int)(kptr[p + 1] - kptr[p]));
  atomicMax(mx, m);
}

__global__ void k_galerkin_T(int64_t N, const int64_t* kptr, const int32_t* kcol, const double* kval,
                             const int32_t* elem_of, const int8_t* comp_of, const double* q1w,
                             const int32_t* cidx, Mesh m, int ndof, int W, int32_t* Tcol,
                             double* Tval, int32_t* Tcnt) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    int32_t* tc = Tcol + p * W;
    double* tv = Tval + p * W;
    int cnt = 0;
    for (int64_t t = kptr[p]; t < kptr[p + 1]; ++t) {
      const int32_t q = kcol[t];
      const double v = kval[t];
      const int eq = elem_of[q];
      const int aq = ndof == 1 ? 0 : comp_of[q];
      for (int c2 = 0; c2 < m.nc; ++c2) {
        const int l = cidx[(int64_t)mesh_of(m, eq, c2) * ndof + aq];
        if (l < 0) continue;
        const double w2 = q1w[(int64_t)c2 * N + q];
        if (w2 == 0.0) continue;
        const double add = v * w2;
        // insert into the row kept sorted by coarse column
        int pos = cnt;
        while (pos > 0 && tc[pos - 1] > l) --pos;
        if (pos > 0 && tc[pos - 1] == l) {
          tv[pos - 1] += add;
        } else {
          for (int u = cnt; u > pos; --u) {
            tc[u] = tc[u - 1];
            tv[u] = tv[u - 1];
          }
          tc[pos] = l;
          tv[pos] = add;
          ++cnt;
        }
      }
    }
    Tcnt[p] = cnt;
  }
}

__global__ void k_galerkin_rows(int n_mesh, Mesh m, int ndof, int64_t N, const int32_t* elem_ptr,
                                const int8_t* comp_of, const double* q1w, const int32_t* cidx,
                                int W, const int32_t* Tcol, const double* Tval, const int32_t* Tcnt,
                                int m0, double* A0) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t ka = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; ka < (int64_t)n_mesh * ndof;
       ka += nw) {
    const int row = cidx[ka];
    if (row < 0) continue;
    const int k = (int)(ka / ndof), a = (int)(ka % ndof);
    int km[3];
    mesh_multi(m, k, km);
    double* out = A0 + (int64_t)row * m0;
    for (int cp = 0; cp < m.nc; ++cp) {
      const int e = elem_around(m, km, cp);
      if (e < 0) continue;
      const int c = (m.nc - 1) - cp;
      for (int p = elem_ptr[e]; p < elem_ptr[e + 1]; ++p) {
        if (ndof > 1 && comp_of[p] != a) continue;
        const double wp = q1w[(int64_t)c * N + p];
        if (wp == 0.0) continue;
        const int cnt = Tcnt[p];
        for (int u = lane; u < cnt; u += 32) {
          const int l = Tcol[(int64_t)p * W + u];
          out[l] += wp * Tval[(int64_t)p * W + u];
        }
        __syncwarp();
      }
    }
  }
}

int pc_galerkin(spnet_pc_s* pc, double* A0) {
  cudaStream_t s = pc->op->stream;
  const Mesh m = mesh_of_pc(pc);
  SPNET_CUDA_TRY(cudaMemsetAsync(A0, 0, sizeof(double) * (size_t)pc->m0 * pc->m0, s));
  if (pc->m0 == 0) return SPNET_OK;
  DevArena tmp;
  tmp.stream = s;
  struct Guard {
    DevArena& a;
    ~Guard() { a.free_all(); }
  } guard{tmp};
  int* mx = nullptr;
  SPNET_TRY(tmp.get(&mx, 1));
  SPNET_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(int), s));
  const int grid = 4 * num_sms();
  note_launch();
  k_galerkin_rowmax<<<grid, 256, 0, s>>>(pc->N, pc->K.ptr, mx);
  int hmx = 0;
  SPNET_CUDA_TRY(cudaMemcpyAsync(&hmx, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  const int W = hmx * pc->nc;
  if (W > GAL_W)
    return fail(SPNET_ERR_UNSUPPORTED, "setup_preconditioner: a row of A is too long for the Galerkin product");
  int32_t *Tcol = nullptr, *Tcnt = nullptr;
  double* Tval = nullptr;
  SPNET_TRY(tmp.get(&Tcol, (size_t)pc->N * W));
  SPNET_TRY(tmp.get(&Tval, (size_t)pc->N * W));
  SPNET_TRY(tmp.get(&Tcnt, pc->N));
  note_launch();
  k_galerkin_T<<<grid, 128, 0, s>>>(pc->N, pc->K.ptr, pc->K.col, pc->K.val, pc->elem_of, pc->comp_of,
                                    pc->q1w, pc->cidx, m, pc->ndof, W, Tcol, Tval, Tcnt);
  const int64_t rows = (int64_t)pc->n_mesh * pc->ndof;
  int blocks = (int)((rows + 7) / 8);
  if (blocks > 16 * num_sms()) blocks = 16 * num_sms();
  note_launch();
  k_galerkin_rows<<<blocks, 256, 0, s>>>(pc->n_mesh, m, pc->ndof, pc->N, pc->elem_ptr, pc->comp_of,
                                         pc->q1w, pc->cidx, W, Tcol, Tval, Tcnt, pc->m0, A0);
  SPNET_CUDA_TRY(cudaGetLastError());
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  return SPNET_OK;
}

}  // namespace spnet
