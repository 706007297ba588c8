// Error reporting, stream-ordered allocation, prefix sums and copies.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "spnet_internal.cuh"

namespace spnet {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

const std::string& last_error() { return g_last_error; }

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int DevArena::alloc(void** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 16;
  cudaError_t e = cudaMallocAsync(p, n, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SPNET_ERR_NO_MEMORY, std::string("device allocation of ") + std::to_string(n) +
                                         " bytes failed: " + cudaGetErrorString(e));
  }
  ptrs.push_back(*p);
  sizes.push_back((int64_t)n);
  bytes += (int64_t)n;
  return SPNET_OK;
}

void DevArena::release(void* p) {
  for (size_t i = 0; i < ptrs.size(); ++i) {
    if (ptrs[i] == p) {
      cudaFreeAsync(p, stream);
      bytes -= sizes[i];
      ptrs.erase(ptrs.begin() + i);
      sizes.erase(sizes.begin() + i);
      return;
    }
  }
}

void DevArena::free_all() {
  for (void* p : ptrs) cudaFreeAsync(p, stream);
  ptrs.clear();
  sizes.clear();
  bytes = 0;
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

void fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s) {
  if (n > 0) {
    note_launch();
    k_fill_i32<<<4 * num_sms(), 256, 0, s>>>(p, n, v);
  }
}

// ---------------------------------------------------------------------------
// launch counting and per-kernel timing (CUDA events on the launching stream)
// ---------------------------------------------------------------------------
static std::atomic<long long> g_launches{0};
static std::atomic<int> g_prof_on{0};
static std::mutex g_prof_mu;
struct ProfRec {
  int id;
  cudaEvent_t a, b;
};
static std::vector<ProfRec> g_prof_pending;
static long long g_prof_n[KID_COUNT];
static double g_prof_ms[KID_COUNT];

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool profiling_on() { return g_prof_on.load(std::memory_order_relaxed) != 0; }
long long launch_count() { return g_launches.load(); }

// events are created once and reused after every drain, so that recording
// costs the host as little as possible and the GPU is not left waiting
static std::vector<cudaEvent_t> g_ev_pool;
static size_t g_ev_next = 0;

static cudaEvent_t pool_event() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_ev_next == g_ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    g_ev_pool.push_back(e);
  }
  return g_ev_pool[g_ev_next++];
}

ProfScope::ProfScope(int id_, cudaStream_t s_) : id(id_), s(s_) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  a = pool_event();
  b = pool_event();
  cudaEventRecord(a, s);
  active = true;
}

ProfScope::~ProfScope() {
  if (!active) return;
  cudaEventRecord(b, s);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_pending.push_back(ProfRec{id, a, b});
}

void profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on.store(on ? 1 : 0);
}

static void profile_drain() {
  std::vector<ProfRec> v;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    v.swap(g_prof_pending);
  }
  for (auto& r : v) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    g_prof_n[r.id] += 1;
    g_prof_ms[r.id] += ms;
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof_pending.empty()) g_ev_next = 0;
}

void profile_read(int id, long long* n, double* ms) {
  profile_drain();
  *n = g_prof_n[id];
  *ms = g_prof_ms[id];
}

void profile_reset() {
  profile_drain();
  for (int i = 0; i < KID_COUNT; ++i) {
    g_prof_n[i] = 0;
    g_prof_ms[i] = 0.0;
  }
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return (double)ms;
}

int copy_in(const void* src, void* dst, size_t bytes, int mem, cudaStream_t s) {
  if (bytes == 0) return SPNET_OK;
  SPNET_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes,
                                 mem == SPNET_MEM_HOST ? cudaMemcpyHostToDevice
                                                       : cudaMemcpyDeviceToDevice,
                                 s));
  return SPNET_OK;
}

int copy_out(const void* src, void* dst, size_t bytes, int mem, cudaStream_t s) {
  if (bytes == 0) return SPNET_OK;
  SPNET_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes,
                                 mem == SPNET_MEM_HOST ? cudaMemcpyDeviceToHost
                                                       : cudaMemcpyDeviceToDevice,
                                 s));
  return SPNET_OK;
}

int check_flags(int* dflags, cudaStream_t s, const char* where) {
  int h = 0;
  SPNET_CUDA_TRY(cudaMemcpyAsync(&h, dflags, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPNET_CUDA_TRY(cudaStreamSynchronize(s));
  if (h == 0) return SPNET_OK;
  std::string w(where);
  if (h & FLAG_NOT_SPD) return fail(SPNET_ERR_NOT_SPD, w + ": non-positive pivot in a local factorisation");
  if (h & FLAG_COARSE_SPD) return fail(SPNET_ERR_NOT_SPD, w + ": non-positive pivot in the coarse matrix");
  if (h & FLAG_ASYM) return fail(SPNET_ERR_BAD_INPUT, w + ": K_II is not symmetric");
  if (h & FLAG_NONFINITE) return fail(SPNET_ERR_BAD_INPUT, w + ": non-finite value");
  if (h & FLAG_OUT_OF_BOX) return fail(SPNET_ERR_BAD_INPUT, w + ": coordinate outside the domain");
  if (h & FLAG_UNSORTED) return fail(SPNET_ERR_BAD_INPUT, w + ": column indices not strictly ascending");
  if (h & FLAG_STAR_BIG) return fail(SPNET_ERR_UNSUPPORTED, w + ": a star exceeds the local solver's capacity");
  if (h & FLAG_POOL) return fail(SPNET_ERR_NO_MEMORY, w + ": factor pool overflow");
  if (h & FLAG_UNCOVERED)
    return fail(SPNET_ERR_BAD_INPUT, w + ": a free dof lies in no star, so B is singular there (take stars at "
                                         "every mesh node, SPNET_STARS_ALL)");
  return fail(SPNET_ERR_BAD_INPUT, w + ": invalid input (index out of range or malformed)");
}

// ---------------------------------------------------------------------------
// exclusive prefix sum: out[i] = sum_{k<i} in[k], out[n] = total
// Three passes over tiles of 4096 items: tile sums, a scan of the tile sums in
// one block, then the tile-local scans.  Deterministic (integer arithmetic).
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t* sh) {
  // inclusive scan across the block (SCAN_T threads) using warp shuffles
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int64_t s = (lane < SCAN_T / 32) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    sh[lane] = s;
  }
  __syncthreads();
  if (wid > 0) v += sh[wid - 1];
  __syncthreads();
  return v;
}

template <class T>
__global__ void k_tile_sums(const T* in, int64_t n, int64_t* tsum) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k)
    if (base + k < n) s += (int64_t)in[base + k];
  int64_t inc = block_incl_scan<T>(s, sh);
  if (threadIdx.x == SCAN_T - 1) tsum[blockIdx.x] = inc;
}

__global__ void k_scan_tiles(int64_t* tsum, int64_t ntiles) {
  __shared__ int64_t sh[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < ntiles; b0 += SCAN_T) {
    int64_t i = b0 + threadIdx.x;
    int64_t v = i < ntiles ? tsum[i] : 0;
    int64_t inc = block_incl_scan<int64_t>(v, sh);
    int64_t c = carry;
    if (i < ntiles) tsum[i] = c + inc - v;  // exclusive
    __syncthreads();
    if (threadIdx.x == SCAN_T - 1) carry = c + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) tsum[ntiles] = carry;
}

template <class T>
__global__ void k_tile_scan(const T* in, int64_t n, const int64_t* tsum, int64_t* out) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t loc[SCAN_ITEMS];
  int64_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    loc[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
    s += loc[k];
  }
  int64_t inc = block_incl_scan<T>(s, sh);
  int64_t run = tsum[blockIdx.x] + inc - s;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = run;
    run += loc[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = tsum[gridDim.x];
}

template <class T>
static int scan_impl(const T* in, int64_t* out, int64_t n, cudaStream_t s, DevArena& mem) {
  int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (ntiles == 0) {
    SPNET_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return SPNET_OK;
  }
  int64_t* tsum = nullptr;
  SPNET_TRY(mem.get(&tsum, ntiles + 1));
  note_launch();
  k_tile_sums<T><<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, n, tsum);
  note_launch();
  k_scan_tiles<<<1, SCAN_T, 0, s>>>(tsum, ntiles);
  note_launch();
  k_tile_scan<T><<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, n, tsum, out);
  SPNET_CUDA_TRY(cudaGetLastError());
  mem.release(tsum);
  return SPNET_OK;
}

int scan_exclusive(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s, DevArena& mem) {
  return scan_impl<int32_t>(in, out, n, s, mem);
}

int scan_exclusive64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, DevArena& mem) {
  return scan_impl<int64_t>(in, out, n, s, mem);
}

}  // namespace spnet
