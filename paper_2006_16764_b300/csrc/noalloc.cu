// Dot products without any device allocation.
//
// Some callers cannot allocate device memory when they need a reduction: a
// host application that has handed all device memory to its own pool
// allocator, a latency-sensitive loop in which the implicit device
// synchronisation of cudaMalloc / cudaFree is not acceptable, or code that
// must not create a tusas handle (tusas_create allocates workspaces). For
// them tusas_multidot_noalloc computes the same deterministic dot products as
// tusas_dot with its per-block partial sums kept in a fixed, file-scope
// device array instead of handle-owned scratch.
//
// The array holds TUSAS_NOALLOC_MAX_K x reduce_blocks() partial sums plus
// TUSAS_NOALLOC_MAX_K results (76 KB of doubles); every GPU that loads the
// library keeps it until the process exits. All calls share it, so calls
// that overlap on the GPU (different streams or host threads) race and must
// be serialised by the caller. Nothing in it has to start at zero: every
// partial sum and result a call reads was written earlier in the same call.
#include <mutex>

#include "../../include/tusas.h"
#include "ops.h"

namespace {

constexpr int kMaxK = TUSAS_NOALLOC_MAX_K;
constexpr int kMaxBlocks = 296;  // tusas::reduce_blocks(), checked at set-up
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kMaxK * kMaxBlocks + kMaxK];

std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device; looked up once
// per device (cudaGetSymbolAddress with that device current) and kept for the
// process, so it goes stale if the device is reset (callers must not reset).
int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TUSAS_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    if (tusas::reduce_blocks() > kMaxBlocks) return TUSAS_EINVAL;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return TUSAS_ECUDA;
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return TUSAS_OK;
}

}  // namespace

extern "C" int tusas_multidot_noalloc(const double* X, long long ld, int k, const double* y, long long n,
                                      double* out, void* stream) {
  if (!out || k < 1 || k > kMaxK || n < 0 || (n > 0 && (!X || !y)) || (k > 1 && ld < n)) return TUSAS_EINVAL;
  if (n == 0) {
    for (int j = 0; j < k; ++j) out[j] = 0.0;
    return TUSAS_OK;
  }
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* partials = scratch;
  double* results = scratch + kMaxK * kMaxBlocks;
  if (tusas::multidot(n, k, X, ld, y, partials, results, st) != cudaSuccess) return TUSAS_ECUDA;
  if (cudaMemcpyAsync(out, results, sizeof(double) * k, cudaMemcpyDeviceToHost, st) != cudaSuccess) return TUSAS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TUSAS_ECUDA;
  return TUSAS_OK;
}
