// Block-diagonal physics-based preconditioner (internal interface).
#pragma once
#include <vector>

#include "ops.h"

namespace tusas {

struct PrecondLevel {
  DevMesh m;
  i64 nn;
  void* st;    // stencils [2 blocks][3^dim offsets][nn], FP32 or FP64
  void* dinv;  // [2][nn]
  void* b;     // right-hand side [2][nn]
  void* x;     // iterate
  void* r_;    // Jacobi-scaled Chebyshev residual
  void* d;     // Chebyshev direction (double buffered with d2)
  void* d2;
  void* res;   // unscaled residual for the restriction
  void* pend;  // after a smoothing: the last Chebyshev direction, not yet added to x (or null)
  double lmax[2];
  int r;       // stencil radius: 1 (3^dim points), 2 on the Q2 node lattice (5 x 5)
};

class Precond {
 public:
  int kind = 0;          // 0 identity, 1 point Jacobi, 2 block Jacobi + GMG
  int fp32 = 1;          // operator / smoother precision
  int cheb_degree = 2, coarse_degree = 10;
  std::vector<PrecondLevel> lv;
  double* gersh_partials = nullptr;  // [blocks][2]
  double* lmax_dev = nullptr;        // [levels][2]
  double* diag = nullptr;            // Q2 point Jacobi: FP64 diagonals of M11, M22 [2][nn]
  size_t bytes = 0;

  // Allocate the hierarchy for the mesh (levels: coarsen by 2 while every
  // element count is even and >= 2, at most `levels`). On a Q2 mesh point
  // Jacobi takes the diagonals from an element pass, and the multigrid starts on
  // the node lattice of spacing h/2 (25-point stencils) above the vertex grid.
  cudaError_t create(const DevMesh& m, int kind, int fp32, int levels, int cheb_degree, int coarse_degree);
  void destroy();
  // Fill the fine stencils of M11 / M22 at the iterate U (Gauss-point
  // coefficients of Eqs. pref2 / preconc2), the Galerkin coarse stencils,
  // D^-1 and the Gershgorin bounds. Synchronises the stream once.
  cudaError_t setup(const ElemCtx& c, double theta, const double* U, const double* Un, cudaStream_t st);
  // z = M^-1 r (FP64 in and out). input_ready: the FP32 multigrid's input for r (the slots
  // of fp32_input) was written by the caller after the last setup, so the narrowing pass is
  // skipped.
  cudaError_t apply(const double* r, double* z, cudaStream_t st, bool input_ready = false);
  // The FP32 multigrid's input slots, for a caller that produces r itself: b = r narrowed to
  // FP32 (narrow<float>) and db = dinv * b, 2 nn floats each. False (and nothing set) for
  // point Jacobi or an FP64 hierarchy.
  bool fp32_input(float** b, float** db, const float** dinv) const;

 private:
  template <typename T>
  cudaError_t setup_t(const ElemCtx& c, double theta, const double* U, const double* Un, cudaStream_t st);
  template <typename T>
  cudaError_t apply_t(const double* r, double* z, cudaStream_t st, bool input_ready);
  template <typename T>
  cudaError_t galerkin_and_bounds(cudaStream_t st);
  // zout: the finest level's post-smoothing writes its result there in FP64 (and sets
  // *zdone) when its last stencil step can take the widening
  template <typename T>
  cudaError_t vcycle(int l, cudaStream_t st, double* zout = nullptr, bool* zdone = nullptr);
  // Chebyshev smoothing of level l; the last step's x += d is left to the next reader of
  // x (residual, prolongation or the FP64 output), which adds lv[l].pend. fold: the last
  // stencil step writes x with that step included instead (a pre-smoothing followed by
  // the residual, a coarse level's smoothing followed by the prolongation)
  template <typename T>
  cudaError_t cheb(int l, bool zero_x, int degree, cudaStream_t st, double* zout = nullptr, bool* zdone = nullptr,
                   bool fold = false);
};

}  // namespace tusas
