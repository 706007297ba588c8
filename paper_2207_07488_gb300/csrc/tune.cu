// The tuner's cache: choices measured at set-up per device and size class.
//
// Three choices are timed on the preconditioner's own data the first time a
// size class is met: the warps per block of the one-vector star solve, the
// lanes per row of the SpMV, and the right-hand sides per warp of the batched
// star solve.  The last two change the order of floating-point sums, so every
// set-up of a class uses the one measured value: a set-up that meets a class
// being measured waits for it, and a class is measured once per process (or
// never, when a cache file saved earlier lists it).  The cache is kept per
// device (name, SM count, compute capability) and can be saved to and loaded
// from a file of lines "device<TAB>kind<TAB>c0,c1,c2,c3<TAB>value".
#include <condition_variable>
#include <cstdio>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

#include "spnet_internal.cuh"

namespace spnet {

namespace {
struct Entry {
  int value = 0;        // the choice (>= 1), or 0 while being measured
};
std::mutex tune_mu;
std::condition_variable tune_cv;
std::map<std::string, Entry> tune_map;  // key: device | kind | class
int64_t tune_measured = 0, tune_reused = 0;

std::string device_key() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p{};
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::ostringstream o;
  for (const char* c = p.name; *c; ++c) o << (*c == '\t' || *c == '\n' ? ' ' : *c);
  o << " sm" << p.multiProcessorCount << " cc" << p.major << p.minor;
  return o.str();
}

std::string key_of(const std::string& dev, int kind, const TuneClass& c) {
  std::ostringstream o;
  o << dev << '\t' << kind << '\t' << c.c[0] << ',' << c.c[1] << ',' << c.c[2] << ',' << c.c[3];
  return o.str();
}
}  // namespace

int tune_begin(int kind, const TuneClass& c, int* value) {
  const std::string key = key_of(device_key(), kind, c);
  std::unique_lock<std::mutex> lk(tune_mu);
  for (;;) {
    auto it = tune_map.find(key);
    if (it == tune_map.end()) {
      tune_map[key] = Entry{};  // this set-up measures the class
      return 0;
    }
    if (it->second.value > 0) {
      *value = it->second.value;
      ++tune_reused;
      return 1;
    }
    tune_cv.wait(lk);  // being measured by another set-up
  }
}

int tune_peek(int kind, const TuneClass& c, int* value) {
  const std::string key = key_of(device_key(), kind, c);
  std::lock_guard<std::mutex> lk(tune_mu);
  auto it = tune_map.find(key);
  if (it == tune_map.end() || it->second.value < 1) return 0;
  *value = it->second.value;
  return 1;
}

void tune_end(int kind, const TuneClass& c, int value) {
  const std::string key = key_of(device_key(), kind, c);
  {
    std::lock_guard<std::mutex> lk(tune_mu);
    if (value > 0) {
      tune_map[key].value = value;
      ++tune_measured;
    } else {
      tune_map.erase(key);  // measuring failed: the next set-up tries again
    }
  }
  tune_cv.notify_all();
}

int half_octave(double x) { return x <= 1.0 ? 0 : (int)std::floor(2.0 * std::log2(x)); }

}  // namespace spnet

using namespace spnet;

extern "C" int spnet_tune_cache_save(const char* path) {
  if (!path) return fail(SPNET_ERR_BAD_INPUT, "spnet_tune_cache_save: null path");
  std::lock_guard<std::mutex> lk(tune_mu);
  std::ofstream f(path);
  if (!f) return fail(SPNET_ERR_BAD_INPUT, std::string("spnet_tune_cache_save: cannot write ") + path);
  for (const auto& kv : tune_map)
    if (kv.second.value > 0) f << kv.first << '\t' << kv.second.value << '\n';
  return f ? SPNET_OK : fail(SPNET_ERR_BAD_INPUT, "spnet_tune_cache_save: write failed");
}

extern "C" int spnet_tune_cache_load(const char* path) {
  if (!path) return fail(SPNET_ERR_BAD_INPUT, "spnet_tune_cache_load: null path");
  std::ifstream f(path);
  if (!f) return fail(SPNET_ERR_BAD_INPUT, std::string("spnet_tune_cache_load: cannot read ") + path);
  std::map<std::string, Entry> add;
  std::string line;
  int ln = 0;
  while (std::getline(f, line)) {
    ++ln;
    if (line.empty()) continue;
    // device \t kind \t c0,c1,c2,c3 \t value
    const size_t a = line.find('\t'), b = a == std::string::npos ? a : line.find('\t', a + 1),
                 c = b == std::string::npos ? b : line.find('\t', b + 1);
    int kind = 0, c0 = 0, c1 = 0, c2 = 0, c3 = 0, v = 0;
    if (c == std::string::npos || line.find('\t', c + 1) != std::string::npos ||
        std::sscanf(line.c_str() + a + 1, "%d", &kind) != 1 ||
        std::sscanf(line.c_str() + b + 1, "%d,%d,%d,%d", &c0, &c1, &c2, &c3) != 4 ||
        std::sscanf(line.c_str() + c + 1, "%d", &v) != 1 || v < 1 || kind < 0 || kind >= TUNE_KINDS)
      return fail(SPNET_ERR_BAD_INPUT, std::string("spnet_tune_cache_load: malformed line ") + std::to_string(ln));
    const TuneClass cls{{c0, c1, c2, c3}};
    add[key_of(line.substr(0, a), kind, cls)].value = v;
  }
  {
    std::lock_guard<std::mutex> lk(tune_mu);
    for (const auto& kv : add) tune_map[kv.first] = kv.second;
  }
  tune_cv.notify_all();
  return SPNET_OK;
}

extern "C" int spnet_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(tune_mu);
  for (auto it = tune_map.begin(); it != tune_map.end();)
    it = it->second.value > 0 ? tune_map.erase(it) : std::next(it);  // keep classes being measured
  tune_measured = tune_reused = 0;
  return SPNET_OK;
}

extern "C" int spnet_tune_counts(int64_t* measured, int64_t* reused) {
  if (!measured || !reused) return fail(SPNET_ERR_BAD_INPUT, "spnet_tune_counts: null argument");
  std::lock_guard<std::mutex> lk(tune_mu);
  *measured = tune_measured;
  *reused = tune_reused;
  return SPNET_OK;
}
