// Device memory of the library's handles, counted on the host.
//
// Every workspace a handle allocates (state vectors, Krylov basis, stored
// linearisation, multigrid hierarchy, adjoint checkpoints) goes through
// dev_malloc / dev_free, which keep the bytes held by the library at once and
// refuse an allocation that would pass the cap set by
// tusas_set_device_bytes_cap. A refused allocation returns
// cudaErrorMemoryAllocation without calling cudaMalloc, exactly like a full
// device, so the allocation-failure paths (TUSAS_ENOMEM) can be exercised
// without exhausting the GPU.
#include <mutex>
#include <unordered_map>

#include "../../include/tusas.h"
#include "ops.h"

namespace tusas {
namespace {
std::mutex g_mu;
std::unordered_map<void*, size_t> g_sizes;
long long g_live = 0;  // bytes held
long long g_cap = 0;   // 0: no cap
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_cap > 0 && g_live + (long long)bytes > g_cap) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  g_sizes[*p] = bytes;
  g_live += (long long)bytes;
  return cudaSuccess;
}

void dev_free(void* p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_sizes.find(p);
    if (it != g_sizes.end()) {
      g_live -= (long long)it->second;
      g_sizes.erase(it);
    }
  }
  cudaFree(p);
}

bool dev_bytes_admit(long long bytes) {
  std::lock_guard<std::mutex> lock(g_mu);
  return g_cap <= 0 || g_live + bytes <= g_cap;
}

}  // namespace tusas

extern "C" int tusas_set_device_bytes_cap(long long bytes) {
  if (bytes < 0) return TUSAS_EINVAL;
  std::lock_guard<std::mutex> lock(tusas::g_mu);
  tusas::g_cap = bytes;
  return TUSAS_OK;
}

extern "C" long long tusas_device_bytes(void) {
  std::lock_guard<std::mutex> lock(tusas::g_mu);
  return tusas::g_live;
}
