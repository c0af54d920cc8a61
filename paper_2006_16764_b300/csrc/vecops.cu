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

// ---- Gram-Schmidt passes of the GMRES orthogonalisation ---------------------------
// Streaming kernels over the basis X_0..X_{k-1} (stride ld) and the new vector w,
// 16-byte loads (pairs of doubles) when n, ld and the pointers allow it. Fixed
// partition of the pairs into GS_BLOCKS contiguous chunks, thread-stride order
// inside a chunk, fixed in-block tree, and one warp per output for the sum of the
// per-block partials: deterministic.
static const int GS_BLOCKS = 148 * 4;
static const int GS_T = 256;

template <int VEC> struct Vec;
template <> struct Vec<1> {
  typedef double T;
  static __device__ __forceinline__ double dot(T a, T b, double acc) { return fma(a, b, acc); }
  static __device__ __forceinline__ T axpy(double c, T x, T y) { return fma(c, x, y); }
  static __device__ __forceinline__ T scale(double c, T x) { return c * x; }
};
template <> struct Vec<2> {
  typedef double2 T;
  static __device__ __forceinline__ double dot(T a, T b, double acc) { return fma(a.y, b.y, fma(a.x, b.x, acc)); }
  static __device__ __forceinline__ T axpy(double c, T x, T y) { return make_double2(fma(c, x.x, y.x), fma(c, x.y, y.y)); }
  static __device__ __forceinline__ T scale(double c, T x) { return make_double2(c * x.x, c * x.y); }
};

// Sum of KM per-thread accumulators over the block into partials[blockIdx.x * 32 + j], j < k.
template <int KM>
__device__ __forceinline__ void gs_block_sum(const double* acc, int k, double* __restrict__ partials) {
  __shared__ double red[GS_T / 32][KM];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < KM; ++j) {
    if (j < k) {
      double v = acc[j];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][j] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < GS_T / 32; ++w) s += red[w][threadIdx.x];
    partials[blockIdx.x * 32 + threadIdx.x] = s;
  }
}

// Unrolled streaming: each thread takes UNR elements of its chunk per trip (stride GS_T) and
// issues all their loads before the arithmetic, so UNR x (k + 1) 16-byte loads are in flight per
// thread. On B300 these passes are bound by the FP64 pipe (2 DFMA per clock per SM: one FMA per
// 8 bytes of basis read runs at most at 4.8 TB/s), so the vector count is a template argument:
// predicated-off FMAs of a rounded-up count still occupy the pipe. KM = exact count when EXACT,
// else an upper bound with k the runtime count.
template <int KM> struct GsUnroll { static const int V = KM <= 4 ? 4 : (KM <= 8 ? 2 : 1); };

// With NORM the ||w||^2 accumulator (kept in acc[KM]) moves to slot k, the column after the dots.
template <int KM, bool NORM>
__device__ __forceinline__ void gs_norm_slot(double* acc, int k) {
  if (NORM && k < KM) {
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j == k) acc[j] = acc[KM];
  }
}

template <int VEC>
__device__ __forceinline__ typename Vec<VEC>::T gs_zero();
template <>
__device__ __forceinline__ double gs_zero<1>() { return 0.0; }
template <>
__device__ __forceinline__ double2 gs_zero<2>() { return make_double2(0.0, 0.0); }

// pass 0: partials[b][j] of X_j . w (j < k), and with NORM partials[b][k] of ||w||^2
template <int KM, int VEC, bool EXACT, bool NORM>
__global__ void __launch_bounds__(GS_T) k_gs_dots(i64 nv, int k, const double* __restrict__ X, i64 ldv,
                                                  const double* __restrict__ w, double* __restrict__ partials) {
  typedef typename Vec<VEC>::T T;
  constexpr int UNR = GsUnroll<KM>::V;
  if (EXACT) k = KM;
  const T* Xv = reinterpret_cast<const T*>(X);
  const T* wv = reinterpret_cast<const T*>(w);
  double acc[KM + 1];
#pragma unroll
  for (int j = 0; j <= KM; ++j) acc[j] = 0.0;
  const i64 chunk = (nv + gridDim.x - 1) / gridDim.x;
  const i64 lo = blockIdx.x * chunk;
  const i64 hi = lo + chunk < nv ? lo + chunk : nv;
  for (i64 i = lo + threadIdx.x; i < hi; i += (i64)GS_T * UNR) {
    T wi[UNR], x[KM][UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const i64 e = i + (i64)u * GS_T;
      wi[u] = e < hi ? wv[e] : gs_zero<VEC>();
#pragma unroll
      for (int j = 0; j < KM; ++j) x[j][u] = ((EXACT || j < k) && e < hi) ? Xv[j * ldv + e] : gs_zero<VEC>();
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
#pragma unroll
      for (int j = 0; j < KM; ++j)
        if (EXACT || j < k) acc[j] = Vec<VEC>::dot(x[j][u], wi[u], acc[j]);
      if (NORM) acc[KM] = Vec<VEC>::dot(wi[u], wi[u], acc[KM]);
    }
  }
  gs_norm_slot<KM, NORM>(acc, k);
  gs_block_sum<NORM ? KM + 1 : KM>(acc, NORM ? k + 1 : k, partials);
}

// pass 1: w -= sum_j c_j X_j, then partials[b][j] of X_j . w (the updated w) and partials[b][k]
// of ||w||^2
template <int KM, int VEC, bool EXACT>
__global__ void __launch_bounds__(GS_T) k_gs_update_dots(i64 nv, int k, const double* __restrict__ X, i64 ldv,
                                                         const double* __restrict__ c, double* __restrict__ w,
                                                         double* __restrict__ partials) {
  typedef typename Vec<VEC>::T T;
  constexpr int UNR = GsUnroll<KM>::V;
  if (EXACT) k = KM;
  const T* Xv = reinterpret_cast<const T*>(X);
  T* wv = reinterpret_cast<T*>(w);
  double cc[KM], acc[KM + 1];
#pragma unroll
  for (int j = 0; j < KM; ++j) {
    cc[j] = (EXACT || j < k) ? -c[j] : 0.0;
    acc[j] = 0.0;
  }
  acc[KM] = 0.0;
  const i64 chunk = (nv + gridDim.x - 1) / gridDim.x;
  const i64 lo = blockIdx.x * chunk;
  const i64 hi = lo + chunk < nv ? lo + chunk : nv;
  for (i64 i = lo + threadIdx.x; i < hi; i += (i64)GS_T * UNR) {
    T wi[UNR], x[KM][UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const i64 e = i + (i64)u * GS_T;
      wi[u] = e < hi ? wv[e] : gs_zero<VEC>();
#pragma unroll
      for (int j = 0; j < KM; ++j) x[j][u] = ((EXACT || j < k) && e < hi) ? Xv[j * ldv + e] : gs_zero<VEC>();
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
#pragma unroll
      for (int j = 0; j < KM; ++j)
        if (EXACT || j < k) wi[u] = Vec<VEC>::axpy(cc[j], x[j][u], wi[u]);
      const i64 e = i + (i64)u * GS_T;
      if (e < hi) wv[e] = wi[u];
#pragma unroll
      for (int j = 0; j < KM; ++j)
        if (EXACT || j < k) acc[j] = Vec<VEC>::dot(x[j][u], wi[u], acc[j]);
      acc[KM] = Vec<VEC>::dot(wi[u], wi[u], acc[KM]);
    }
  }
  gs_norm_slot<KM, true>(acc, k);
  gs_block_sum<KM + 1>(acc, k + 1, partials);
}

// The FP32 multigrid's input for the vector element(s) e of pass 2 (GsNarrow).
__device__ __forceinline__ void gs_narrow_store(const GsNarrow& nw, i64 e, double o) {
  const float b = narrow<float>(o);
  nw.b[e] = b;
  nw.db[e] = nw.dinv[e] * b;
}
__device__ __forceinline__ void gs_narrow_store(const GsNarrow& nw, i64 e, double2 o) {
  const float2 b = make_float2(narrow<float>(o.x), narrow<float>(o.y));
  const float2 d = reinterpret_cast<const float2*>(nw.dinv)[e];
  reinterpret_cast<float2*>(nw.b)[e] = b;
  reinterpret_cast<float2*>(nw.db)[e] = make_float2(d.x * b.x, d.y * b.y);
}

// pass 2: w = (w - sum_j c_j X_j) s[0], and the FP32 multigrid's input for w if nw.b is set
template <int KM, int VEC, bool EXACT>
__global__ void __launch_bounds__(GS_T) k_gs_update_scale(i64 nv, int k, const double* __restrict__ X, i64 ldv,
                                                          const double* __restrict__ c, const double* __restrict__ s,
                                                          double* __restrict__ w, GsNarrow nw) {
  typedef typename Vec<VEC>::T T;
  constexpr int UNR = GsUnroll<KM>::V;
  if (EXACT) k = KM;
  const T* Xv = reinterpret_cast<const T*>(X);
  T* wv = reinterpret_cast<T*>(w);
  double cc[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) cc[j] = (EXACT || j < k) ? -c[j] : 0.0;
  const double sc = s[0];
  const i64 chunk = (nv + gridDim.x - 1) / gridDim.x;
  const i64 lo = blockIdx.x * chunk;
  const i64 hi = lo + chunk < nv ? lo + chunk : nv;
  for (i64 i = lo + threadIdx.x; i < hi; i += (i64)GS_T * UNR) {
    T wi[UNR], x[KM][UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const i64 e = i + (i64)u * GS_T;
      wi[u] = e < hi ? wv[e] : gs_zero<VEC>();
#pragma unroll
      for (int j = 0; j < KM; ++j) x[j][u] = ((EXACT || j < k) && e < hi) ? Xv[j * ldv + e] : gs_zero<VEC>();
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
#pragma unroll
      for (int j = 0; j < KM; ++j)
        if (EXACT || j < k) wi[u] = Vec<VEC>::axpy(cc[j], x[j][u], wi[u]);
      const i64 e = i + (i64)u * GS_T;
      if (e < hi) {
        const T o = Vec<VEC>::scale(sc, wi[u]);
        wv[e] = o;
        if (nw.b) gs_narrow_store(nw, e, o);
      }
    }
  }
}

// pass 3: w -= sum_j c_j X_j (no reduction; the first half of pass 1 for long cycles)
template <int KM, int VEC, bool EXACT>
__global__ void __launch_bounds__(GS_T) k_gs_update(i64 nv, int k, const double* __restrict__ X, i64 ldv,
                                                    const double* __restrict__ c, double* __restrict__ w) {
  typedef typename Vec<VEC>::T T;
  constexpr int UNR = GsUnroll<KM>::V;
  if (EXACT) k = KM;
  const T* Xv = reinterpret_cast<const T*>(X);
  T* wv = reinterpret_cast<T*>(w);
  double cc[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) cc[j] = (EXACT || j < k) ? -c[j] : 0.0;
  const i64 chunk = (nv + gridDim.x - 1) / gridDim.x;
  const i64 lo = blockIdx.x * chunk;
  const i64 hi = lo + chunk < nv ? lo + chunk : nv;
  for (i64 i = lo + threadIdx.x; i < hi; i += (i64)GS_T * UNR) {
    T wi[UNR], x[KM][UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const i64 e = i + (i64)u * GS_T;
      wi[u] = e < hi ? wv[e] : gs_zero<VEC>();
#pragma unroll
      for (int j = 0; j < KM; ++j) x[j][u] = ((EXACT || j < k) && e < hi) ? Xv[j * ldv + e] : gs_zero<VEC>();
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
#pragma unroll
      for (int j = 0; j < KM; ++j)
        if (EXACT || j < k) wi[u] = Vec<VEC>::axpy(cc[j], x[j][u], wi[u]);
      const i64 e = i + (i64)u * GS_T;
      if (e < hi) wv[e] = wi[u];
    }
  }
}

// the fused update + dots of pass 1 keeps the KM loaded basis values in registers: up to 16
static const int GS_FUSED_MAX = 16;

// pass 0: dots; 1: update + dots + norm (fused up to GS_FUSED_MAX vectors); 2: update + scale;
// 3: update alone; 4: dots + norm (3 then 4 is pass 1 for long cycles)
template <int KM, int VEC, bool EXACT>
static void gs_kernel(int pass, i64 nv, int k, const double* X, i64 ldv, const double* c, const double* s, double* w,
                      double* partials, cudaStream_t st, GsNarrow nw) {
  if (pass == 0) {
    k_gs_dots<KM, VEC, EXACT, false><<<GS_BLOCKS, GS_T, 0, st>>>(nv, k, X, ldv, w, partials);
  } else if (pass == 1) {
    if constexpr (KM <= GS_FUSED_MAX) k_gs_update_dots<KM, VEC, EXACT><<<GS_BLOCKS, GS_T, 0, st>>>(nv, k, X, ldv, c, w, partials);
  } else if (pass == 2) {
    k_gs_update_scale<KM, VEC, EXACT><<<GS_BLOCKS, GS_T, 0, st>>>(nv, k, X, ldv, c, s, w, nw);
  } else if (pass == 3) {
    k_gs_update<KM, VEC, EXACT><<<GS_BLOCKS, GS_T, 0, st>>>(nv, k, X, ldv, c, w);
  } else {
    k_gs_dots<KM, VEC, EXACT, true><<<GS_BLOCKS, GS_T, 0, st>>>(nv, k, X, ldv, w, partials);
  }
}

// 16-byte loads: one instantiation per vector count up to 30 (the longest GMRES cycle); the
// scalar-load fallback takes rounded counts.
static cudaError_t gs_launch_vec2(int pass, i64 n, int k, const double* X, i64 ld, const double* c,
                                  const double* s, double* w, double* partials, cudaStream_t st, GsNarrow nw) {
  const i64 nv = n / 2, ldv = ld / 2;
  switch (k) {
#define TUSAS_GS_K(K) \
  case K:             \
    gs_kernel<K, 2, true>(pass, nv, k, X, ldv, c, s, w, partials, st, nw); \
    break;
    TUSAS_GS_K(1) TUSAS_GS_K(2) TUSAS_GS_K(3) TUSAS_GS_K(4) TUSAS_GS_K(5) TUSAS_GS_K(6) TUSAS_GS_K(7)
    TUSAS_GS_K(8) TUSAS_GS_K(9) TUSAS_GS_K(10) TUSAS_GS_K(11) TUSAS_GS_K(12) TUSAS_GS_K(13) TUSAS_GS_K(14)
    TUSAS_GS_K(15) TUSAS_GS_K(16) TUSAS_GS_K(17) TUSAS_GS_K(18) TUSAS_GS_K(19) TUSAS_GS_K(20) TUSAS_GS_K(21)
    TUSAS_GS_K(22) TUSAS_GS_K(23) TUSAS_GS_K(24) TUSAS_GS_K(25) TUSAS_GS_K(26) TUSAS_GS_K(27) TUSAS_GS_K(28)
    TUSAS_GS_K(29) TUSAS_GS_K(30)
#undef TUSAS_GS_K
    default:
      gs_kernel<31, 2, false>(pass, nv, k, X, ldv, c, s, w, partials, st, nw);
  }
  count_launches(1);
  return cudaGetLastError();
}

static cudaError_t gs_launch_scalar(int pass, i64 n, int k, const double* X, i64 ld, const double* c,
                                    const double* s, double* w, double* partials, cudaStream_t st, GsNarrow nw) {
  if (k <= 4)
    gs_kernel<4, 1, false>(pass, n, k, X, ld, c, s, w, partials, st, nw);
  else if (k <= 8)
    gs_kernel<8, 1, false>(pass, n, k, X, ld, c, s, w, partials, st, nw);
  else if (k <= 16)
    gs_kernel<16, 1, false>(pass, n, k, X, ld, c, s, w, partials, st, nw);
  else
    gs_kernel<31, 1, false>(pass, n, k, X, ld, c, s, w, partials, st, nw);
  count_launches(1);
  return cudaGetLastError();
}

int gs_blocks() { return GS_BLOCKS; }

cudaError_t gs_pass(int pass, i64 n, int k, const double* X, i64 ld, const double* c, const double* s, double* w,
                    double* partials, double* out, cudaStream_t st, GsNarrow nw) {
  if (k < 1 || k > 31 || pass < 0 || pass > 2) return cudaErrorInvalidValue;
  if (pass != 2) nw = GsNarrow();
  if (nw.b && (!nw.db || !nw.dinv)) return cudaErrorInvalidValue;
  // the 16-byte path stores the FP32 outputs as 8-byte pairs
  const bool nw_ok = !nw.b || (((uintptr_t)nw.b | (uintptr_t)nw.db | (uintptr_t)nw.dinv) % 8) == 0;
  const bool vec = n % 2 == 0 && ld % 2 == 0 && ((uintptr_t)X % 16) == 0 && ((uintptr_t)w % 16) == 0 && nw_ok;
  if (pass == 1 && k > GS_FUSED_MAX) {
    // the fused update + dots would spill with this many vectors in registers: update, then
    // dots + norm
    cudaError_t e = vec ? gs_launch_vec2(3, n, k, X, ld, c, s, w, partials, st, nw)
                        : gs_launch_scalar(3, n, k, X, ld, c, s, w, partials, st, nw);
    if (e != cudaSuccess) return e;
    return vec ? gs_launch_vec2(4, n, k, X, ld, c, s, w, partials, st, nw)
               : gs_launch_scalar(4, n, k, X, ld, c, s, w, partials, st, nw);
  }
  cudaError_t e = vec ? gs_launch_vec2(pass, n, k, X, ld, c, s, w, partials, st, nw)
                      : gs_launch_scalar(pass, n, k, X, ld, c, s, w, partials, st, nw);
  if (e != cudaSuccess || pass != 0) return e;
  k_reduce_partials<<<1, 32 * k, 0, st>>>(GS_BLOCKS, k, 32, partials, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tusas
