// Per-device host state of the launchers: the dynamic shared-memory limit of each kernel (a
// function attribute applies to one device's context; it is raised when a launch needs more than
// the limit set so far), the SM count and the shared-memory budgets, all kept per device under a
// mutex, so several host threads and several GPUs may launch.
#include <map>
#include <mutex>
#include <utility>

#include "doa_internal.cuh"

namespace doa {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
std::map<std::pair<int, const void *>, int> g_attr_bytes;   // (device, kernel) -> the limit set
int g_sms[kMaxDevices] = {};
SmemLimits g_smem[kMaxDevices] = {};

}  // namespace

cudaError_t ensure_smem_attr(const void *func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mutex);
  auto it = g_attr_bytes.find({dev, func});
  if (it != g_attr_bytes.end() && it->second >= bytes) return cudaSuccess;   // raised only, never lowered
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) g_attr_bytes[{dev, func}] = bytes;
  return e;
}

int device_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_sms[dev] <= 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_sms[dev] = n > 0 ? n : 1;
  }
  return g_sms[dev];
}

SmemLimits device_smem_limits() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SmemLimits{49152, 49152, 0};
  std::lock_guard<std::mutex> lock(g_mutex);
  SmemLimits &l = g_smem[dev];
  if (l.per_sm <= 0) {
    int sm = 0, blk = 0, res = 0;
    cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&res, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    l = SmemLimits{sm > 0 ? sm : 49152, blk > 0 ? blk : 49152, res > 0 ? res : 0};
  }
  return l;
}

}  // namespace doa
