// Status codes, the per-thread error message and the device status word.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "umma.cuh"

namespace nedmft {

namespace {
thread_local std::string g_last_error;

// One status word per device (a file-scope device variable exists once on
// every device that loads the library).
__device__ int g_status_word;

constexpr int kMaxDevices = 64;
int* g_status_addr[kMaxDevices] = {nullptr};
std::mutex g_status_mu;
}  // namespace

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return set_error(NEDMFT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {
std::atomic<bool> g_instr_on{false};
std::atomic<bool> g_instr_timing{false};
std::atomic<long long> g_launches{0};
std::mutex g_instr_mu;
struct Slot { cudaEvent_t a, b; double flops, bytes; };
std::vector<Slot> g_slots;
size_t g_slot_used = 0;
}  // namespace

void instr_count() {
  if (g_instr_on.load(std::memory_order_relaxed)) g_launches.fetch_add(1, std::memory_order_relaxed);
}
bool instr_timing() { return g_instr_timing.load(std::memory_order_relaxed); }
int instr_begin(cudaStream_t st) {
  if (!instr_timing()) return -1;
  std::lock_guard<std::mutex> lk(g_instr_mu);
  if (g_slot_used == g_slots.size()) {
    Slot s{};
    if (cudaEventCreate(&s.a) != cudaSuccess || cudaEventCreate(&s.b) != cudaSuccess) return -1;
    g_slots.push_back(s);
  }
  int k = (int)g_slot_used++;
  g_slots[k].flops = 0.0;
  if (cudaEventRecord(g_slots[k].a, st) != cudaSuccess) return -1;
  return k;
}
void instr_end(int slot, cudaStream_t st, double flops, double bytes) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_instr_mu);
  cudaEventRecord(g_slots[slot].b, st);
  g_slots[slot].flops = flops;
  g_slots[slot].bytes = bytes;
}

int* device_status_ptr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_status_mu);
  if (!g_status_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
    g_status_addr[dev] = static_cast<int*>(p);
  }
  return g_status_addr[dev];
}

namespace {
std::mutex g_attr_mu;
std::vector<std::pair<const void*, int>> g_attr_done[kMaxDevices];  // (kernel, bytes) per device
int g_sm_count[kMaxDevices] = {0};
}  // namespace

int ensure_dyn_smem(const void* kern, int bytes) {
  int dev = 0;
  NED_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(NEDMFT_ECUDA, "device %d beyond the library's table", dev);
  std::lock_guard<std::mutex> lk(g_attr_mu);
  for (const auto& e : g_attr_done[dev])
    if (e.first == kern && e.second >= bytes) return NEDMFT_OK;
  NED_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  g_attr_done[dev].emplace_back(kern, bytes);
  return NEDMFT_OK;
}

namespace {
struct ClusterFit { const void* kern; int block, smem, clusters; };
std::vector<ClusterFit> g_cluster_fit[kMaxDevices];
}  // namespace

int max_active_clusters(const void* kern, int block, int smem_bytes, int* out) {
  int dev = 0;
  NED_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(NEDMFT_ECUDA, "device %d beyond the library's table", dev);
  std::lock_guard<std::mutex> lk(g_attr_mu);
  for (const auto& f : g_cluster_fit[dev])
    if (f.kern == kern && f.block == block && f.smem == smem_bytes) {
      *out = f.clusters;
      return NEDMFT_OK;
    }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  NED_CUDA(cudaOccupancyMaxActiveClusters(&n, kern, &cfg));
  if (n < 1) return set_error(NEDMFT_ECUDA, "no cluster of two CTAs with %d bytes of shared memory fits", smem_bytes);
  g_cluster_fit[dev].push_back({kern, block, smem_bytes, n});
  *out = n;
  return NEDMFT_OK;
}

int device_sm_count(int* out) {
  int dev = 0;
  NED_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(NEDMFT_ECUDA, "device %d beyond the library's table", dev);
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (!g_sm_count[dev]) NED_CUDA(cudaDeviceGetAttribute(&g_sm_count[dev], cudaDevAttrMultiProcessorCount, dev));
  *out = g_sm_count[dev];
  return NEDMFT_OK;
}

}  // namespace nedmft

using namespace nedmft;

extern "C" const char* nedmft_status_string(int status) {
  switch (status) {
    case NEDMFT_OK: return "ok";
    case NEDMFT_EINVAL: return "invalid argument";
    case NEDMFT_ENOMEM: return "workspace too small";
    case NEDMFT_ECUDA: return "CUDA runtime error";
    case NEDMFT_ESINGULAR: return "pivot below threshold (matrix singular to working precision)";
    case NEDMFT_ETIMEOUT: return "bounded device wait expired";
    case NEDMFT_ENOTCONV: return "not converged within max_iter";
    default: return "unknown status";
  }
}

extern "C" const char* nedmft_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* nedmft_version(void) { return "nedmft-gb300 0.1 (sm_103a)"; }

extern "C" int nedmft_check_status(void* stream) {
  int* p = device_status_ptr();
  if (!p) return set_error(NEDMFT_ECUDA, "cannot locate the device status word");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int host = 0;
  NED_CUDA(cudaMemcpyAsync(&host, p, sizeof(int), cudaMemcpyDeviceToHost, s));
  NED_CUDA(cudaStreamSynchronize(s));
  if (host != DS_OK) {
    NED_CUDA(cudaMemsetAsync(p, 0, sizeof(int), s));
    NED_CUDA(cudaStreamSynchronize(s));
  }
  if (host == DS_SINGULAR) return set_error(NEDMFT_ESINGULAR, "a Gauss-Jordan pivot fell below the threshold");
  if (host == DS_TIMEOUT) return set_error(NEDMFT_ETIMEOUT, "a bounded device wait expired");
  return NEDMFT_OK;
}

extern "C" int nedmft_instrument(int enable, int timing) {
  std::lock_guard<std::mutex> lk(g_instr_mu);
  g_instr_on = enable != 0;
  g_instr_timing = enable != 0 && timing != 0;
  g_launches = 0;
  g_slot_used = 0;
  return NEDMFT_OK;
}

extern "C" int nedmft_instrument_read(int64_t* launches, int64_t* timed_launches, double* timed_ms,
                                      double* timed_flops, double* timed_bytes) {
  std::lock_guard<std::mutex> lk(g_instr_mu);
  double ms = 0.0, fl = 0.0, by = 0.0;
  for (size_t k = 0; k < g_slot_used; ++k) {
    NED_CUDA(cudaEventSynchronize(g_slots[k].b));
    float t = 0.0f;
    NED_CUDA(cudaEventElapsedTime(&t, g_slots[k].a, g_slots[k].b));
    ms += t;
    fl += g_slots[k].flops;
    by += g_slots[k].bytes;
  }
  if (launches) *launches = g_launches.load();
  if (timed_launches) *timed_launches = (int64_t)g_slot_used;
  if (timed_ms) *timed_ms = ms;
  if (timed_flops) *timed_flops = fl;
  if (timed_bytes) *timed_bytes = by;
  return NEDMFT_OK;
}

extern "C" int nedmft_set_wait_limit(double seconds, void* stream) {
  if (!(seconds >= 0.0 && seconds <= 60.0))
    return set_error(NEDMFT_EINVAL, "set_wait_limit: %g s outside [0, 60]", seconds);
  return umma_set_wait_ns((uint64_t)(seconds * 1e9), static_cast<cudaStream_t>(stream));
}

extern "C" int nedmft_wait_selftest(void* stream) {
  int* p = device_status_ptr();
  if (!p) return set_error(NEDMFT_ECUDA, "cannot locate the device status word");
  return umma_wait_selftest(p, static_cast<cudaStream_t>(stream));
}
