// Host-side launch interface of the tusas-b300 kernels (internal to the library).
#pragma once
#include <utility>
#include <cuda_runtime.h>

#include "common.cuh"
#include "element.cuh"

namespace tusas {

// kernels launched by the library (instrumentation)
void count_launches(long long n);
long long launches();

// Device allocations of the handles, counted against the cap of
// tusas_set_device_bytes_cap (cudaErrorMemoryAllocation past it, without
// calling cudaMalloc). dev_bytes_admit: whether `bytes` more would fit.
cudaError_t dev_malloc(void** p, size_t bytes);
void dev_free(void* p);
bool dev_bytes_admit(long long bytes);
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}

// M_DIAG (Q2 only): the diagonals of the preconditioner blocks M11, M22.
enum ElemMode { M_RES = 0, M_RES_LIN = 1, M_JV = 2, M_JTV = 3, M_DEPS = 4, M_PREV_T = 5, M_OLD = 6, M_DIAG = 7 };

// 1D tables of the biquadratic element with the 3-point Gauss rule (g Gauss
// point, a local node): B = Lagrange values, G = physical derivatives (1/h);
// BW = h w_g B, GW = h w_g G (test side, w_g the unit-interval weights);
// BB = h w_g B^2, GG = h w_g G^2 (diagonal of mass / stiffness forms);
// xg = Gauss points in [0, 1].
struct Q2Tab {
  double B[3][3], G[3][3], BW[3][3], GW[3][3], BB[3][3], GG[3][3], xg[3];
};

struct ElemCtx {
  DevMesh m;
  DevPhys P;
  Scales S;
  LinScale K;   // scaled linearisation of the Q1 tangent / adjoint passes
  LinScale Ku;  // unit factors (Q2 passes)
  PwConst pw_elem, pw_res3, pw_q2;  // pointwise constants per kernel family (gradient units, factors)
  Q2Tab q2;
  int ntx, nty, ntz;  // tiles per axis
  int nlin;           // linearisation coefficients per Gauss point
};

// One tile-colour launch of an element pass. Colours after the first are programmatic
// dependents of the previous colour: their CTAs may start on the SMs its last wave frees,
// because the kernels touch nothing the previous colour writes until their node sums, where
// they wait for it (griddepcontrol.wait) and read the sums past L1.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_colour(void (*kernel)(KArgs...), unsigned blocks, unsigned threads, size_t smem,
                                 cudaStream_t st, bool dependent, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

void elem_ctx_init(ElemCtx& c, const DevMesh& m, const DevPhys& P);
// Doubles of the linearisation store for this mesh / model.
size_t elem_lin_doubles(const ElemCtx& c);
// Element-tile pass: out = (mode-dependent) assembled vector; out is zeroed
// (or set to `init`) first, then the 2^dim tile colours accumulate in a fixed
// order. `phold`: nodal (phi^n - phi^{n-1})/dt when the Eq. (theta) estimate is used.
cudaError_t elem_run(int mode, const ElemCtx& c, const double* U, const double* Un, const double* V, double* out,
                     double* lin, cudaStream_t st, const double* init = nullptr, const double* phold = nullptr);
// The same pass on a 2D Q2 box (out already zeroed or initialised by elem_run).
cudaError_t q2_run(int mode, const ElemCtx& c, const double* U, const double* Un, const double* V, double* out,
                   double* lin, cudaStream_t st, const double* phold);
void q2_tables(Q2Tab& T, double h);
// Stencils of the preconditioner blocks of a triquadratic box: [2][125][nn] on its node
// lattice and, if stv, [2][27][nv] on its element-vertex grid (T = float or double).
template <typename T>
cudaError_t q2h_stencil_fill(const ElemCtx& c, const double* U, const double* Un, T* st, T* stv, cudaStream_t s);
// The same pass on a 3D box of triquadratic (Q2) hexes with the 3 x 3 x 3 Gauss rule.
cudaError_t q2h_run(int mode, const ElemCtx& c, const double* U, const double* Un, const double* V, double* out,
                    double* lin, cudaStream_t st, const double* phold);
// 25-point stencils [2][25][nodes] of the preconditioner blocks of a Q2 box on its node
// lattice, at the iterate U with U^n (T = float or double).
template <typename T>
cudaError_t q2_stencil_fill(const ElemCtx& c, const double* U, const double* Un, T* st, cudaStream_t s);

// ---- FP64 vector kernels (deterministic) ----------------------------------
// y = a*x + y
cudaError_t vaxpy(i64 n, double a, const double* x, double* y, cudaStream_t st);
// z = x + a*y   (a read from device memory when ad != nullptr: z = x + (*ad)*y)
cudaError_t vxpay(i64 n, const double* x, double a, const double* ad, const double* y, double* z, cudaStream_t st);
// y = (y - x) * (*ainv)   (finite-difference quotient, ainv on device)
cudaError_t vfdq(i64 n, const double* x, double* y, const double* ainv, cudaStream_t st);
// y = x * (*s) (s on device, optionally inverted)
cudaError_t vscale_dev(i64 n, const double* x, double* y, const double* s, int invert, cudaStream_t st);
cudaError_t vcopy(i64 n, const double* x, double* y, cudaStream_t st);
// y *= a
cudaError_t vscal(i64 n, double a, double* y, cudaStream_t st);
cudaError_t vfill(i64 n, double v, double* y, cudaStream_t st);

// out[j] = sum_i X_j[i] * y[i] for j < k, X_j = X + j*ld; partials has
// k * reduce_blocks() doubles. Deterministic (fixed partition and order).
int reduce_blocks();
cudaError_t multidot(i64 n, int k, const double* X, i64 ld, const double* y, double* partials, double* out,
                     cudaStream_t st);
// y -= sum_j c[j] X_j (c on device, k entries), optionally scaled: if accum_c
// != nullptr, accum_c[j] += c[j] as well.
cudaError_t multi_axpy(i64 n, int k, const double* X, i64 ld, const double* c, double* y, double* accum_c,
                       cudaStream_t st);
// y -= sum_j c[j] X_j fused with the deterministic norm: *out_norm2 = ||y||^2
cudaError_t multi_axpy_norm(i64 n, int k, const double* X, i64 ld, const double* c, double* y, double* partials,
                            double* out_norm2, cudaStream_t st);
// Gram-Schmidt passes of the GMRES orthogonalisation over X_0..X_{k-1} (k <= 31) and w,
// deterministic; partials holds gs_blocks() x 32 doubles; c, s and out are device arrays:
//   pass 0: out[j] = X_j . w (reduced)
//   pass 1: w -= sum_j c[j] X_j, then the per-block partial sums of X_j . w in partials[b][j]
//           and of ||w||^2 in partials[b][k], left for the caller to reduce (b < gs_blocks())
//   pass 2: w = (w - sum_j c[j] X_j) s[0]; with nw.b set it also writes nw.b = w narrowed
//           to FP32 (narrow<float>) and nw.db = nw.dinv * nw.b, the FP32 multigrid's input
//           for w (Precond::fp32_input), n elements each
struct GsNarrow {
  float* b = nullptr;
  float* db = nullptr;
  const float* dinv = nullptr;
};
int gs_blocks();
cudaError_t gs_pass(int pass, i64 n, int k, const double* X, i64 ld, const double* c, const double* s, double* w,
                    double* partials, double* out, cudaStream_t st, GsNarrow nw = GsNarrow());
// x = sum_j c[j] X_j + x (c on host memory passed by value through a device array)
cudaError_t multi_comb(i64 n, int k, const double* X, i64 ld, const double* c, double* x, cudaStream_t st);

}  // namespace tusas
