/*
 * tusas-b300: C-ABI of the B300 (sm_103a) hot path of the fully implicit
 * phase-field method of Ghosh, Newman and Francois, "Tusas: a fully implicit
 * parallel approach for coupled phase-field equations" (arXiv 2006.16764).
 *
 * The library evaluates, on one GPU, the discrete residual F(U) of the coupled
 * phase-field / solute (or dimensionless temperature) system on a structured
 * box of Q1 quadrilaterals or hexahedra, or Q2 quadrilaterals (Sec. 2.1.1,
 * Eqs. pf2, conc2, gs, jat, with the theta-method of Eqs. dpf, dc, theta), its
 * Jacobian action (finite difference, Eq. JFmatvec, or an exact tangent), the
 * transposed action, the block-diagonal preconditioner of Eq. (pre), a
 * Newton-Krylov time step (Sec. 2.2, 2.3) and a discrete adjoint through a
 * sequence of steps.
 *
 * Conventions for every entry point:
 *   - vectors are FP64 arrays of length 2*N_nodes, field-major
 *     [phi(0..N_nodes-1) ; u(0..N_nodes-1)], node index i + nnx (j + nny k) with
 *     nnx = order nx + 1, nny = order ny + 1 (tusas_mesh);
 *   - vector pointers are caller-owned DEVICE memory of the handle's device
 *     unless an entry point says otherwise; the library never frees them;
 *   - work is enqueued on the handle's stream (tusas_set_stream) and is
 *     asynchronous unless the entry point says that it synchronises;
 *   - every call returns TUSAS_OK (0) or a negative code and never aborts the
 *     process; tusas_last_error() gives a one-line description.
 */
#ifndef TUSAS_H
#define TUSAS_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TUSAS_OK = 0,
  TUSAS_EINVAL = -1,     /* bad mesh, parameters, pointer or size            */
  TUSAS_ECUDA = -2,      /* a CUDA runtime call failed                        */
  TUSAS_ENOMEM = -3,     /* device allocation failed or exceeded the cap      */
  TUSAS_ENOCONV = -4,    /* Newton / GMRES / line search did not converge     */
  TUSAS_ENONFINITE = -5  /* a NaN or Inf appeared in a residual norm          */
};

/* Structured box of nx x ny (x nz) Lagrange elements of size h; dim 2 (nz = 0)
 * or 3 (Sec. 2.1.1). order 0 or 1: Q1 elements with the 2^dim-point Gauss
 * rule, node (i,j,k) at (x0 + i h, y0 + j h, z0 + k h). order 2: biquadratic
 * Q2 elements with the 3 x 3 Gauss rule (2D only; the higher-order elements of
 * the tip-velocity study, Sec. 4.1), node (i,j) at (x0 + i h/2, y0 + j h/2),
 * (2 nx + 1)(2 ny + 1) nodes; their multigrid (precond 2) starts on the node
 * lattice of spacing h/2 (25-point stencils) and coarsens to the element
 * vertices; tusas_create returns TUSAS_EINVAL for order 2 in 3D. Nodes are
 * numbered x fastest in every case. */
typedef struct tusas_mesh {
  int dim;
  int nx, ny, nz;
  double h;
  double x0, y0, z0;
  int order;
} tusas_mesh;

/* Model and solver parameters, nondimensional (Sec. 4.2: W0 = tau0 = 1).
 * model 0: pure metal (Karma-Rappel phi + temperature u, k must be 1);
 * model 1: dilute binary alloy (Sec. 4.2, Eqs. pf2..jat). */
typedef struct tusas_params {
  int model;
  double W0, tau0, eps4, lam, D, k;
  double lT, Vp, zT;     /* frozen gradient G4 = (x_last - zT - Vp t)/lT, model 1, lT != 0 */
  double theta;          /* theta-method weight in [0, 1] (Eqs. dpf, dc): 1 backward Euler, 1/2 Crank-Nicolson */
  int phihat_form;       /* theta < 1: phihat of the solute source and antitrapping current is
                            1: (phi^{n+1} - phi^n)/dt (second order at theta = 1/2), or
                            0: the estimate of Eq. (theta), theta (phi^{n+1}-phi^n)/dt + (1-theta)(phi^n-phi^{n-1})/dt */
  int jat_normalised;    /* 1: antitrapping along grad(phi)/|grad(phi)|, 0: along grad(phi) */
  int time_form;         /* 0: tau0 B a^2 (phi - phi^n)/dt; 1: tau0 ([B a^2 phi]^{n+1} - [..]^n)/dt */
  int jvp_mode;          /* Newton-Krylov Jacobian action: 0 finite difference, 1 exact tangent */
  int precond;           /* 0 none, 1 point Jacobi, 2 block Jacobi with geometric multigrid */
  int smoother_fp32;     /* multigrid operators, smoother and coarse levels in FP32 (1) or FP64 (0) */
  int gmres_restart;     /* Krylov vectors per cycle, 1..30 */
  int gmres_maxit;       /* GMRES iterations per Newton iteration (a truncated solve is still a Newton direction) */
  int newton_maxit;
  double newton_rtol, newton_atol;
  double eta0, eta_min, eta_max, gamma, omega;   /* forcing terms, Eqs. force1..forcing */
  int mg_levels, cheb_degree, coarse_degree, linesearch_max;
} tusas_params;

/* Statistics of one tusas_step. */
typedef struct tusas_stats {
  int converged;
  int newton_its;
  int gmres_its;
  int linesearch_halvings;
  int residual_evals;      /* evaluations of F over the whole mesh          */
  int jv_evals;            /* Jacobian actions over the whole mesh          */
  double fnorm0, fnorm;    /* ||F|| at the first and last Newton iterate     */
  int gmres_per_newton[32];
} tusas_stats;

typedef struct tusas_handle tusas_handle;

/* Create a handle on the current CUDA device: validates mesh and parameters
 * and allocates the handle's workspaces (state, Krylov basis, linearisation
 * store, multigrid hierarchy). Returns TUSAS_EINVAL, TUSAS_ENOMEM or
 * TUSAS_ECUDA on failure with *out = NULL. */
int tusas_create(const tusas_mesh* mesh, const tusas_params* params, tusas_handle** out);

/* Free every workspace of the handle (synchronises its stream). NULL is a no-op. */
void tusas_destroy(tusas_handle* h);

/* Stream for all later work (a cudaStream_t; NULL = legacy default stream). */
int tusas_set_stream(tusas_handle* h, void* cuda_stream);

/* Replace the parameters (same rules as tusas_create; the mesh is fixed). */
int tusas_set_params(tusas_handle* h, const tusas_params* params);

/* Number of unknowns 2*(nx+1)(ny+1)(nz+1) of the handle's mesh. */
long long tusas_ndofs(const tusas_handle* h);

/* Set the state U^n (copied; host or device pointer, any memory the CUDA
 * runtime can address), its time t^n and the step dt used by later calls.
 * Synchronises. */
int tusas_set_state(tusas_handle* h, const double* U, double t, double dt);

/* Set U^{n-1} (host or device pointer) for the Eq. (theta) estimate
 * (theta < 1, phihat_form 0). tusas_set_state resets it to U^n; tusas_step
 * shifts it. Synchronises. */
int tusas_set_history(tusas_handle* h, const double* Unm1);

/* Copy the current state into U (host or device pointer). Synchronises. */
int tusas_get_state(tusas_handle* h, double* U);

/* Current time t^n of the state. */
double tusas_time(const tusas_handle* h);

/* F(U) of Eqs. (pf2)/(conc2) with the theta-method of Eqs. (dpf)/(dc) and the
 * stored U^n (and U^{n-1}), t^n, dt:
 * Galerkin residual on the Q1 mesh with the 2^dim-point Gauss rule. U and F
 * are device vectors (may not alias). Deterministic: bitwise identical on
 * repeated calls. */
int tusas_residual(tusas_handle* h, const double* U, double* F);

/* Exact Jacobian action Jv = F'(U) v (Sec. 2.2, the operator that Eq.
 * JFmatvec approximates). Builds the pointwise linearisation at U, then
 * applies it. U, v, Jv device vectors (Jv may not alias U or v). */
int tusas_jvp(tusas_handle* h, const double* U, const double* v, double* Jv);

/* Finite-difference action (F(U + eps v) - F(U))/eps of Eq. (JFmatvec) with
 * eps = sqrt((1 + ||U||) 2^-52)/||v||. Device vectors; Jv = 0 when v = 0. */
int tusas_jvp_fd(tusas_handle* h, const double* U, const double* v, double* Jv);

/* Transposed action JTw = F'(U)^T w (the adjoint of tusas_jvp). */
int tusas_jtvp(tusas_handle* h, const double* U, const double* w, double* JTw);

/* (dF/dU^n)^T w at U, with the stored U^n: the coupling of consecutive time
 * steps in a discrete adjoint (time terms, and for theta < 1 the level-n
 * spatial terms weighted 1 - theta). TUSAS_EINVAL for theta < 1 with
 * phihat_form 0, where F also depends on U^{n-1}. */
int tusas_jtvp_prev(tusas_handle* h, const double* U, const double* w, double* out);

/* dF/dp at U for parameter `which` (0 = eps4, the anisotropy of Eq. gs), through the time
 * term and the flux at both time levels of the theta-method. TUSAS_EINVAL for theta < 1 with
 * phihat_form 0. */
int tusas_dFdp(tusas_handle* h, const double* U, int which, double* dF);

/* Build the preconditioner of Eq. (pre) (blocks of Eqs. pref2 / preconc2)
 * at the iterate U with the stored U^n and dt. */
int tusas_precond_setup(tusas_handle* h, const double* U);

/* z = M^-1 r with the preconditioner of the last tusas_precond_setup:
 * identity, point Jacobi, or one multigrid V-cycle per diagonal block.
 * r and z are FP64 device vectors and may not alias. */
int tusas_precond_apply(tusas_handle* h, const double* r, double* z);

/* One time step of size dt (backward Euler at theta = 1, the theta-method of Eqs. dpf / dc
 * otherwise): solve F(U; U^n) = 0 by Newton-Krylov
 * (Sec. 2.2/2.3: right-preconditioned restarted GMRES, forcing terms,
 * backtracking line search) from U = U^n, then U^n <- U, t^n <- t^n + dt.
 * Synchronises; fills *stats if non-NULL. On TUSAS_ENOCONV the state is
 * left unchanged. */
int tusas_step(tusas_handle* h, tusas_stats* stats);

/* Forward sweep for a discrete adjoint (no counterpart in the paper, whose
 * solver needs only F and J v): set the state to U0 (host or device) at t0,
 * take nsteps steps of size dt with tusas_step (any theta; phihat_form 1 when theta < 1), and record
 * U_0, U_c, U_2c, ... (c = ckpt_every) in handle-owned device memory. The
 * state becomes U_N. *total (if non-NULL) sums the step statistics.
 * Synchronises. Returns the first failing step's code. */
int tusas_forward(tusas_handle* h, const double* U0, double t0, double dt, int nsteps, int ckpt_every,
                  tusas_stats* total);

/* Discrete adjoint of the last tusas_forward for S = w^T U_N (w a device
 * vector): J_N^T lam_N = w, J_n^T lam_n = -(dF_{n+1}/dU_n)^T lam_{n+1},
 * each solved by right-preconditioned FGMRES on J^T (same preconditioner,
 * which is symmetric) to ||r|| <= adj_rtol ||rhs|| within max(gmres_maxit,
 * 1000) iterations (the forward steps keep gmres_maxit); the states are
 * recomputed segment by segment from the checkpoints (deterministic, so they
 * equal the forward's). Returns dS/d eps4 = -sum_n lam_n^T dF_n/d eps4 in
 * *grad_eps4 (host); if grad_dir != NULL, (dS/dU_0) . d0 for the device
 * direction d0 (NULL gives 0); if g0 != NULL, dS/dU_0 = -(dF_1/dU_0)^T lam_1
 * (device). The state is restored to U_N. stats->gmres_its counts the adjoint
 * Krylov iterations, stats->newton_its the adjoint solves. Synchronises;
 * TUSAS_ENOCONV if a solve misses its tolerance. */
int tusas_adjoint(tusas_handle* h, const double* w, const double* d0, double* grad_eps4, double* grad_dir,
                  double* g0, double adj_rtol, tusas_stats* stats);

/* Solid fraction S = int (1 + phi_h)/2 over the box (no counterpart in the
 * paper: the functional whose discrete adjoint gradient tusas_adjoint gives):
 * S = w^T U + |Omega|/2 with w = [(1/2) int psi_i ; 0], the exact integral of
 * the Q1 (or Q2, Simpson node weights) interpolant of phi. If U != NULL
 * (device vector), *S (host) receives S and the call synchronises; if
 * w != NULL (device vector of 2 N_nodes doubles, not aliasing U), it receives
 * the weights, which are dS/dU and the right-hand side of the adjoint. The
 * handle computes the weights once (one vector of device memory).
 * TUSAS_EINVAL if both U and w are NULL, or U is given without S. */
int tusas_solid_fraction(tusas_handle* h, const double* U, double* S, double* w);

/* Deterministic FP64 dot product x . y of n doubles (device vectors); the
 * result is written to *result (host pointer). Synchronises. */
int tusas_dot(tusas_handle* h, const double* x, const double* y, long long n, double* result);

/* ---- Instrumentation (no counterpart in the paper) ------------------------
 * Device time per kernel class, measured with CUDA events recorded on the
 * handle's stream around each operator application inside the library. */
enum {
  TUSAS_T_RESIDUAL = 0,      /* F(U) element-tile pass                         */
  TUSAS_T_RESIDUAL_LIN = 1,  /* F(U) + pointwise linearisation store           */
  TUSAS_T_JV = 2,            /* Jacobian action (stored tangent or FD sequence)*/
  TUSAS_T_ADJOINT = 3,       /* J^T w, (dF/dU^n)^T w, dF/d eps4                */
  TUSAS_T_PC_APPLY = 4,      /* preconditioner application                     */
  TUSAS_T_PC_SETUP = 5,      /* stencil fill, Galerkin coarsening, bounds      */
  TUSAS_T_ORTHO = 6,         /* GMRES classical Gram-Schmidt (twice) + norm    */
  TUSAS_NTIMERS = 7
};
/* Enable (1) or disable (0) the timers; either resets them. */
int tusas_timers(tusas_handle* h, int enable);
/* Accumulated milliseconds and counts per class (host arrays of
 * TUSAS_NTIMERS entries). Synchronises the stream. */
int tusas_get_timers(tusas_handle* h, double* ms, long long* counts);
/* Number of CUDA kernels this library has launched in this process. */
long long tusas_kernel_launches(void);
/* Throughput of dependent FMA chains on the current device (all SMs, 8
 * independent chains per thread): FP64 and FP32 FLOP/s (an FMA counts 2).
 * Allocates and frees a small device buffer. Synchronises the device. */
int tusas_fma_peak(double* fp64_flops, double* fp32_flops);

/* ---- Reductions without device allocation (no counterpart in the paper) ----
 * For callers that cannot allocate device memory at the point where they need
 * a reduction (all device memory handed to their own pool allocator, a loop
 * that cannot afford the implicit synchronisation of cudaMalloc/cudaFree, or
 * code that must not create a handle, which allocates workspaces):
 * out[j] = X_j . y for j < k, X_j = X + j*ld, n doubles each (device
 * vectors), with the same deterministic partition and summation order as
 * tusas_dot, so k = 1 returns tusas_dot's value. Results go to the host array
 * out[k]. The partial sums live in a fixed device array of the library
 * (TUSAS_NOALLOC_MAX_K x 296 + TUSAS_NOALLOC_MAX_K doubles, about 76 KB per
 * GPU, held until the process exits); nothing is allocated or freed. The
 * first call on a device looks up that array's address (cudaGetSymbolAddress
 * with the device current) and keeps it for the process. A cudaDeviceReset of
 * that device reloads the library's module and makes the kept address stale:
 * do not call this entry point on a device after resetting it.
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller. Works on `stream` (a cudaStream_t, NULL = legacy
 * default) and synchronises it. Returns TUSAS_EINVAL for k < 1,
 * k > TUSAS_NOALLOC_MAX_K, n < 0, null pointers or ld < n when k > 1;
 * TUSAS_ECUDA if a CUDA call fails. */
#define TUSAS_NOALLOC_MAX_K 32
int tusas_multidot_noalloc(const double* X, long long ld, int k, const double* y, long long n, double* out,
                           void* stream);

/* ---- Device memory accounting (no counterpart in the paper) --------------
 * The library counts the device bytes its handles hold (state vectors, Krylov
 * basis, linearisation store, multigrid hierarchy, checkpoints; not the
 * fixed array of tusas_multidot_noalloc). With a cap set (bytes > 0) an
 * allocation that would pass it fails as if the device were full: the call
 * returns TUSAS_ENOMEM and frees what it had allocated. tusas_create checks
 * its vectors and Krylov basis against the cap before any CUDA call. 0
 * removes the cap (the default); TUSAS_EINVAL for bytes < 0. Process-wide. */
int tusas_set_device_bytes_cap(long long bytes);
/* Device bytes held by the library's handles at this moment. */
long long tusas_device_bytes(void);

/* Description of the last error on this handle (never NULL). */
const char* tusas_last_error(const tusas_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* TUSAS_H */
