// Allocation-free restriction r_c = R_0 r (the set-up already holds the structure).
//
// The restriction needs scratch for the Q1-weighted corner sums of r on every
// element.  spnet_pc_restrict takes that scratch from the preconditioner's own
// device memory; spnet_pc_restrict_static takes it from a fixed array that is
// part of the library image, so the call itself never allocates: it serves
// callers whose device memory is all reserved up front by another allocator,
// and loops that must not enter cudaMalloc (which can synchronise the device
// and take an unbounded time).
#include <mutex>

#include "spnet_internal.cuh"

namespace spnet {

// Scratch of spnet_pc_restrict_static: corner sums, n_elem * 2^d * ndof doubles
// at most (2 MiB).  Every GPU that loads the library holds it until exit.
constexpr int64_t STATIC_CORNER_SUMS = int64_t(1) << 18;
static __device__ __align__(256) double g_corner_sums[STATIC_CORNER_SUMS];

// device address of the array, looked up once per device with that device current
// (in host code the name g_corner_sums is a host-side stand-in, not a device address)
static double* g_corner_sums_addr[64] = {};
static std::mutex g_corner_sums_mu;

// `dev` is the preconditioner's device; it must be the current one, since the
// symbol lookup and the launches act on the current device
static int corner_sums_address(int dev, double** out) {
  int cur = 0;
  SPNET_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != dev)
    return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_restrict_static: the preconditioner's device (" +
                                         std::to_string(dev) + ") is not the current device (" +
                                         std::to_string(cur) + ")");
  if (dev < 0 || dev >= 64) return fail(SPNET_ERR_UNSUPPORTED, "spnet_pc_restrict_static: device id >= 64");
  std::lock_guard<std::mutex> lk(g_corner_sums_mu);
  if (!g_corner_sums_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_corner_sums);
    if (e != cudaSuccess)
      return fail(SPNET_ERR_CUDA, std::string("spnet_pc_restrict_static: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
    g_corner_sums_addr[dev] = static_cast<double*>(p);
  }
  *out = g_corner_sums_addr[dev];
  return SPNET_OK;
}

// one warp per element: corner sums of r read in free order through perm
template <int NC, int ND>
__global__ void __launch_bounds__(256) k_corner_sums_gather(int n_elem, int64_t N,
                                                            const int32_t* __restrict__ elem_ptr,
                                                            const int32_t* __restrict__ perm,
                                                            const int8_t* __restrict__ comp_of,
                                                            const double* __restrict__ q1w,
                                                            const double* __restrict__ r_free,
                                                            double* __restrict__ sums) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = gwarp; e < n_elem; e += nwarps) {
    double acc[NC * ND];
#pragma unroll
    for (int t = 0; t < NC * ND; ++t) acc[t] = 0.0;
    for (int i = elem_ptr[e] + lane; i < elem_ptr[e + 1]; i += 32) {
      const double v = r_free[perm[i]];
      const int a = ND == 1 ? 0 : comp_of[i];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double wv = q1w[(int64_t)c * N + i] * v;
#pragma unroll
        for (int b = 0; b < ND; ++b)
          if (b == a) acc[c * ND + b] += wv;
      }
    }
#pragma unroll
    for (int t = 0; t < NC * ND; ++t) {
      double v = acc[t];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sums[e * (NC * ND) + t] = v;
    }
  }
}

__global__ void k_restrict_sums(int n_mesh, Mesh m, int ndof, const double* __restrict__ sums,
                                const int32_t* __restrict__ cidx, double* __restrict__ rc) {
  for (int64_t ka = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ka < (int64_t)n_mesh * ndof;
       ka += (int64_t)gridDim.x * blockDim.x) {
    const int ci = cidx[ka];
    if (ci < 0) continue;
    const int k = (int)(ka / ndof), a = (int)(ka % ndof);
    int km[3];
    mesh_multi(m, k, km);
    double s = 0.0;
    for (int cp = 0; cp < m.nc; ++cp) {
      const int e = elem_around(m, km, cp);
      if (e < 0) continue;
      s += sums[((int64_t)e * m.nc + (m.nc - 1 - cp)) * ndof + a];
    }
    rc[ci] = s;
  }
}

}  // namespace spnet

using namespace spnet;

extern "C" int spnet_pc_restrict_static(spnet_pc_t pc, const double* r, double* rc) {
  cudaGetLastError();
  if (!pc || !r || !rc) return fail(SPNET_ERR_BAD_INPUT, "spnet_pc_restrict_static: null argument");
  const int64_t need = (int64_t)pc->n_elem * pc->nc * pc->ndof;
  if (need > STATIC_CORNER_SUMS)
    return fail(SPNET_ERR_UNSUPPORTED,
                "spnet_pc_restrict_static: the mesh needs " + std::to_string(need) +
                    " corner sums, more than the static scratch of " + std::to_string(STATIC_CORNER_SUMS) +
                    " (n_elem * 2^d * ndof)");
  double* sums = nullptr;
  SPNET_TRY(corner_sums_address(pc->op->device, &sums));
  if (pc->m0 == 0) return SPNET_OK;
  cudaStream_t s = pc->op->stream;
  const Mesh m = mesh_of_pc(pc);
  const int grid = 4 * num_sms();
  note_launch();
  if (pc->nc == 4 && pc->ndof == 1)
    k_corner_sums_gather<4, 1><<<grid, 256, 0, s>>>(pc->n_elem, pc->N, pc->elem_ptr, pc->perm, pc->comp_of, pc->q1w, r, sums);
  else if (pc->nc == 8 && pc->ndof == 1)
    k_corner_sums_gather<8, 1><<<grid, 256, 0, s>>>(pc->n_elem, pc->N, pc->elem_ptr, pc->perm, pc->comp_of, pc->q1w, r, sums);
  else if (pc->nc == 4)
    k_corner_sums_gather<4, 3><<<grid, 256, 0, s>>>(pc->n_elem, pc->N, pc->elem_ptr, pc->perm, pc->comp_of, pc->q1w, r, sums);
  else
    k_corner_sums_gather<8, 3><<<grid, 256, 0, s>>>(pc->n_elem, pc->N, pc->elem_ptr, pc->perm, pc->comp_of, pc->q1w, r, sums);
  note_launch();
  const int64_t n = (int64_t)pc->n_mesh * pc->ndof;
  k_restrict_sums<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pc->n_mesh, m, pc->ndof, sums, pc->cidx, rc);
  SPNET_CUDA_TRY(cudaGetLastError());
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  return SPNET_OK;
}
