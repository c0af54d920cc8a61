// Shared device-side definitions of the tusas-b300 library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tusas {

typedef long long i64;

// Structured box of Lagrange elements of order 1 (Q1) or 2 (Q2, 2D only): node
// (i,j,k) at x0 + i h / order, index i + nnx (j + nny k), nnx = order nx + 1.
struct DevMesh {
  int dim;
  int order;
  int nx, ny, nz;        // elements per axis (nz = 0 in 2D)
  int nnx, nny, nnz;     // nodes per axis (nnz = 1 in 2D)
  i64 nn;                // number of nodes
  i64 ne;                // number of elements
  double h, x0, y0, z0;
};

// Pointwise physics constants (Sec. 4.2 model in Karma-Rappel units).
struct DevPhys {
  int model;             // 0 pure metal, 1 dilute alloy
  int time_form;         // 0 c^{n+1}(phi - phi^n)/dt, 1 difference of products
  int jat_norm;          // antitrapping direction: 1 unit normal, 0 grad(phi)
  double W0, tau0, eps4, lam, D, k;
  double lT, Vp, zT;
  double dt, idt;        // time step and its reciprocal
  double t_new;          // t^{n+1}, used by the frozen gradient
  int has_g4;            // model 1 and lT != 0
  // theta-method: spatial terms weighted theta at n+1 and (1 - theta) at n
  double theta;
  double thW2, thD;      // theta W0^2, theta D
  double dphat;          // d phihat / d phi^{n+1}: 1/dt, or theta/dt with the Eq. (theta) estimate
  int phihat_old;        // 1: phihat includes (1 - theta)(phi^n - phi^{n-1})/dt
};

// Tile shape of the element kernels: one thread per element.
template <int DIM> struct Tile;
template <> struct Tile<2> { static const int X = 16, Y = 8, Z = 1; };
template <> struct Tile<3> { static const int X = 8, Y = 4, Z = 4; };

// Tile of the triquadratic (Q2 hex) kernels: one warp per element, the lanes
// taking the 27 Gauss points (and the 27 element nodes in the transposed pass).
struct Q2HexTile { static const int X = 4, Y = 2, Z = 2; };

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Narrowing of FP64 inputs to the fill / smoother precision. To FP32 it runs on the integer
// pipe instead of the FP64 unit (B300 converts 64-bit floats at the FP64 rate, 2 per clock per
// SM): the binary32 result takes the sign, the exponent re-biased from 1023 to 127 and the top
// 23 of the 52 mantissa bits (rounding toward zero, relative error below 2^-23). Magnitudes
// below the binary32 normal range give a signed zero, above it (or NaN) an infinity; the
// states and residuals narrowed here are finite and of order one or zero.
__device__ __forceinline__ float f32_from_f64_rz(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  const unsigned mant = (unsigned)(b >> 29) & 0x7fffffu;
  const unsigned r = e <= 0 ? sign : (e >= 255 ? (sign | 0x7f800000u) : (sign | ((unsigned)e << 23) | mant));
  return __uint_as_float(r);
}
template <typename T>
__device__ __forceinline__ T narrow(double x);
template <>
__device__ __forceinline__ double narrow<double>(double x) { return x; }
template <>
__device__ __forceinline__ float narrow<float>(double x) { return f32_from_f64_rz(x); }


}  // namespace tusas
