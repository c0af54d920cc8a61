// FMA-chain throughput probe (instrumentation): the FP64 and FP32 peaks that
// the roofline of the FP64-bound element kernels is measured against.
#include <atomic>

#include "../../include/tusas.h"
#include "ops.h"

namespace tusas {

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches += n; }
long long launches() { return g_launches.load(); }

template <typename T>
__global__ void k_fma_chain(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static double run_chain(int sms, int iters, double* best) {
  const int threads = 256, blocks = sms * 8;
  T* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(T) * threads * blocks) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  *best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_fma_chain<T><<<blocks, threads>>>(buf, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double fl = 2.0 * 8.0 * iters * (double)threads * blocks;
    if (ms > 0 && fl / (ms * 1e-3) > *best) *best = fl / (ms * 1e-3);
  }
  count_launches(3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  return cudaGetLastError() == cudaSuccess ? 0.0 : -1.0;
}

}  // namespace tusas

extern "C" long long tusas_kernel_launches(void) { return tusas::launches(); }

extern "C" int tusas_fma_peak(double* fp64_flops, double* fp32_flops) {
  if (!fp64_flops || !fp32_flops) return TUSAS_EINVAL;
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return TUSAS_ECUDA;
  if (tusas::run_chain<double>(p.multiProcessorCount, 2048, fp64_flops) < 0) return TUSAS_ECUDA;
  if (tusas::run_chain<float>(p.multiProcessorCount, 32768, fp32_flops) < 0) return TUSAS_ECUDA;
  return TUSAS_OK;
}
