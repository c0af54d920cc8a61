// FP64 vector kernels of the Krylov / Newton path (GMRES inner products run on
// the GPU, Sec. 4.3). Reductions are deterministic: a fixed partition of the
// index range into reduce_blocks() chunks, a fixed in-block tree, and a
// second pass in which one warp per output sums the per-block partials (lane l
// takes partials l, l + 32, ... in order, then a fixed shuffle tree).
// The multi-dot splits the k vectors into groups of 4 over a second grid axis
// (one block per chunk and group), which keeps few registers per thread and
// many blocks per SM; each partial is still the chunk's sum in thread-stride
// order and fixed in-block tree, whatever the grouping.
#include "ops.h"

namespace tusas {

static const int VT = 256;  // threads per block of the vector kernels

static int grid_for(i64 n) {
  i64 g = (n + VT - 1) / VT;
  const i64 cap = 148 * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

__global__ void k_axpy(i64 n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}
__global__ void k_xpay(i64 n, const double* __restrict__ x, double a, const double* __restrict__ ad,
                       const double* __restrict__ y, double* __restrict__ z) {
  const double s = ad ? *ad : a;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    z[i] = fma(s, y[i], x[i]);
}
__global__ void k_fdq(i64 n, const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ ainv) {
  const double s = *ainv;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    y[i] = (y[i] - x[i]) * s;
}
__global__ void k_scale_dev(i64 n, const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ s,
                            int invert) {
  const double f = invert ? 1.0 / *s : *s;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    y[i] = x[i] * f;
}
__global__ void k_scal(i64 n, double a, double* __restrict__ y) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) y[i] *= a;
}
__global__ void k_fill(i64 n, double v, double* __restrict__ y) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) y[i] = v;
}

cudaError_t vaxpy(i64 n, double a, const double* x, double* y, cudaStream_t st) {
  {
    k_axpy<<<grid_for(n), VT, 0, st>>>(n, a, x, y);
    count_launches(1);
  }
  return cudaGetLastError();
}
cudaError_t vxpay(i64 n, const double* x, double a, const double* ad, const double* y, double* z, cudaStream_t st) {
  {
    k_xpay<<<grid_for(n), VT, 0, st>>>(n, x, a, ad, y, z);
    count_launches(1);
  }
  return cudaGetLastError();
}
cudaError_t vfdq(i64 n, const double* x, double* y, const double* ainv, cudaStream_t st) {
  {
    k_fdq<<<grid_for(n), VT, 0, st>>>(n, x, y, ainv);
    count_launches(1);
  }
  return cudaGetLastError();
}
cudaError_t vscale_dev(i64 n, const double* x, double* y, const double* s, int invert, cudaStream_t st) {
  {
    k_scale_dev<<<grid_for(n), VT, 0, st>>>(n, x, y, s, invert);
    count_launches(1);
  }
  return cudaGetLastError();
}
cudaError_t vcopy(i64 n, const double* x, double* y, cudaStream_t st) {
  return cudaMemcpyAsync(y, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
}
cudaError_t vscal(i64 n, double a, double* y, cudaStream_t st) {
  {
    k_scal<<<grid_for(n), VT, 0, st>>>(n, a, y);
    count_launches(1);
  }
  return cudaGetLastError();
}
cudaError_t vfill(i64 n, double v, double* y, cudaStream_t st) {
  {
    k_fill<<<grid_for(n), VT, 0, st>>>(n, v, y);
    count_launches(1);
  }
  return cudaGetLastError();
}

// ---- deterministic multi-dot ------------------------------------------------
static const int RB = 296;  // reduction blocks: 2 per SM
int reduce_blocks() { return RB; }

template <int JG>
__global__ void __launch_bounds__(VT) k_multidot(i64 n, int k, const double* __restrict__ X, i64 ld,
                                                 const double* __restrict__ y, double* __restrict__ partials,
                                                 int km) {
  __shared__ double red[VT / 32][JG];
  const int j0 = blockIdx.y * JG;
  const int kg = k - j0 < JG ? k - j0 : JG;  // vectors of this group
  double acc[JG];
#pragma unroll
  for (int j = 0; j < JG; ++j) acc[j] = 0.0;
  const i64 chunk = (n + gridDim.x - 1) / gridDim.x;
  const i64 lo = blockIdx.x * chunk;
  const i64 hi = lo + chunk < n ? lo + chunk : n;
  const double* Xg = X + j0 * ld;
  for (i64 i = lo + threadIdx.x; i < hi; i += VT) {
    const double yi = y[i];
#pragma unroll
    for (int j = 0; j < JG; ++j)
      if (j < kg) acc[j] = fma(Xg[j * ld + i], yi, acc[j]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < JG; ++j) {
    if (j < kg) {
      double v = acc[j];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][j] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < kg) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < VT / 32; ++w) s += red[w][threadIdx.x];
    partials[blockIdx.x * (i64)km + j0 + threadIdx.x] = s;
  }
}

// out[j] = sum_b partials[b km + j]: warp j, fixed per-lane order and shuffle tree (blockDim = 32 k)
__global__ void k_reduce_partials(int nb, int k, int km, const double* __restrict__ partials, double* __restrict__ out) {
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (j >= k) return;
  double s = 0.0;
  for (int b = lane; b < nb; b += 32) s += partials[b * (i64)km + j];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) out[j] = s;
}

cudaError_t multidot(i64 n, int k, const double* X, i64 ld, const double* y, double* partials, double* out,
                     cudaStream_t st) {
  if (k <= 0 || k > 32) return cudaErrorInvalidValue;
  // partials[b km + j]: km = 1 for a single dot, else 32 (fixed stride for every k)
  const int km = k == 1 ? 1 : 32;
  if (k == 1) {
    k_multidot<1><<<dim3(RB, 1), VT, 0, st>>>(n, k, X, ld, y, partials, km);
  } else {
    k_multidot<4><<<dim3(RB, (k + 3) / 4), VT, 0, st>>>(n, k, X, ld, y, partials, km);
  }
  count_launches(1);
  {
    k_reduce_partials<<<1, 32 * k, 0, st>>>(RB, k, km, partials, out);
    count_launches(1);
  }
  return cudaGetLastError();
}

template <int KM>
__global__ void __launch_bounds__(VT) k_multi_axpy(i64 n, int k, const double* __restrict__ X, i64 ld,
                                                   const double* __restrict__ c, double sign, double* __restrict__ y) {
  double cc[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) cc[j] = j < k ? sign * c[j] : 0.0;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double v = y[i];
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) v = fma(cc[j], X[j * ld + i], v);
    y[i] = v;
  }
}

__global__ void k_add_small(int k, const double* __restrict__ c, double* __restrict__ acc) {
  if (threadIdx.x < k) acc[threadIdx.x] += c[threadIdx.x];
}

static cudaError_t multi_axpy_sign(i64 n, int k, const double* X, i64 ld, const double* c, double sign, double* y,
                                   cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  if (k > 32) return cudaErrorInvalidValue;
  const int g = grid_for(n);
  if (k <= 4)
    {
      k_multi_axpy<4><<<g, VT, 0, st>>>(n, k, X, ld, c, sign, y);
      count_launches(1);
    }
  else if (k <= 8)
    {
      k_multi_axpy<8><<<g, VT, 0, st>>>(n, k, X, ld, c, sign, y);
      count_launches(1);
    }
  else if (k <= 16)
    {
      k_multi_axpy<16><<<g, VT, 0, st>>>(n, k, X, ld, c, sign, y);
      count_launches(1);
    }
  else
    {
      k_multi_axpy<32><<<g, VT, 0, st>>>(n, k, X, ld, c, sign, y);
      count_launches(1);
    }
  return cudaGetLastError();
}

cudaError_t multi_axpy(i64 n, int k, const double* X, i64 ld, const double* c, double* y, double* accum_c,
                       cudaStream_t st) {
  cudaError_t e = multi_axpy_sign(n, k, X, ld, c, -1.0, y, st);
  if (e != cudaSuccess || accum_c == nullptr) return e;
  {
    k_add_small<<<1, 32, 0, st>>>(k, c, accum_c);
    count_launches(1);
  }
  return cudaGetLastError();
}

// y -= sum_j c[j] X_j and out_norm2 = ||y||^2 (after the update), deterministic.
template <int KM>
__global__ void __launch_bounds__(VT) k_multi_axpy_norm(i64 n, int k, const double* __restrict__ X, i64 ld,
                                                        const double* __restrict__ c, double* __restrict__ y,
                                                        double* __restrict__ partials) {
  __shared__ double red[VT / 32];
  double cc[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) cc[j] = j < k ? -c[j] : 0.0;
  const i64 chunk = (n + gridDim.x - 1) / gridDim.x;
  const i64 lo = blockIdx.x * chunk;
  const i64 hi = lo + chunk < n ? lo + chunk : n;
  double acc = 0.0;
  for (i64 i = lo + threadIdx.x; i < hi; i += VT) {
    double v = y[i];
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) v = fma(cc[j], X[j * ld + i], v);
    y[i] = v;
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < VT / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

cudaError_t multi_axpy_norm(i64 n, int k, const double* X, i64 ld, const double* c, double* y, double* partials,
                            double* out_norm2, cudaStream_t st) {
  if (k < 1 || k > 32) return cudaErrorInvalidValue;
  const int nb = 148 * 8;  // one partial per block; partials holds RB * 32 >= nb doubles
  if (k <= 4) {
    k_multi_axpy_norm<4><<<nb, VT, 0, st>>>(n, k, X, ld, c, y, partials);
  } else if (k <= 8) {
    k_multi_axpy_norm<8><<<nb, VT, 0, st>>>(n, k, X, ld, c, y, partials);
  } else if (k <= 16) {
    k_multi_axpy_norm<16><<<nb, VT, 0, st>>>(n, k, X, ld, c, y, partials);
  } else {
    k_multi_axpy_norm<32><<<nb, VT, 0, st>>>(n, k, X, ld, c, y, partials);
  }
  count_launches(1);
  k_reduce_partials<<<1, 32, 0, st>>>(nb, 1, 1, partials, out_norm2);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t multi_comb(i64 n, int k, const double* X, i64 ld, const double* c, double* x, cudaStream_t st) {
  return multi_axpy_sign(n, k, X, ld, c, 1.0, x, st);
}

}  // namespace tusas
