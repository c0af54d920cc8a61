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

}  // namespace tusas
