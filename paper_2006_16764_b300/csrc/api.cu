// C-ABI entry points (include/tusas.h): handle, state, operator calls and the
// Newton-Krylov time step of Sec. 2.2 / 2.3. The host loop only sees scalars
// (norms, the Hessenberg column); every vector operation runs in the
// library's kernels on the handle's stream.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/tusas.h"
#include "ops.h"
#include "precond.h"

using tusas::i64;

struct tusas_handle {
  tusas_mesh mesh;
  tusas_params prm;
  tusas::DevMesh dm;
  tusas::ElemCtx ec;
  cudaStream_t st = nullptr;
  int device = 0;
  i64 nn = 0, N = 0;
  double t = 0.0, dt = 0.0;
  bool have_state = false;
  double *Un = nullptr, *U = nullptr, *F = nullptr, *Ft = nullptr, *dU = nullptr, *Ut = nullptr, *tmp = nullptr,
         *tmp2 = nullptr;
  double *lin = nullptr, *lin_t = nullptr;
  size_t lin_n = 0;
  double *V = nullptr, *Z = nullptr;
  int m = 0;  // restart length the basis was allocated for
  double* partials = nullptr;
  double* sc = nullptr;  // device scalars: [0..63] h1, [64..127] h2, [128..191] y, [192..] misc
  double* hess = nullptr;  // GMRES Hessenberg H [(m+1) x m], Givens cs, sn [m], g [m+1], status [4]
  double* st_host = nullptr;      // mapped pinned copy of the GMRES status, written by k_arnoldi_givens
  double* st_host_dev = nullptr;  // its device address
  cudaEvent_t ev_st = nullptr;    // recorded after k_arnoldi_givens
  tusas::Precond pc;
  bool pc_ready = false;
  // the Krylov vector whose FP32 multigrid input the last Gram-Schmidt pass wrote (consumed by
  // the next preconditioner apply of that vector), or null
  const double* pc_input_for = nullptr;
  std::string err;
  // instrumentation: CUDA-event pairs per kernel class
  bool timers_on = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> marks;
  double t_ms[TUSAS_NTIMERS] = {};
  long long t_cnt[TUSAS_NTIMERS] = {};
  // discrete adjoint: checkpoints of the last recorded forward sweep
  std::vector<double*> ckpt;   // states U_0, U_c, U_2c, ...
  std::vector<double*> seg;    // recomputed states of one segment
  double* lam = nullptr;       // adjoint variable
  double* lam_rhs = nullptr;
  double* Ufinal = nullptr;
  int fw_steps = 0, fw_every = 0;
  double fw_t0 = 0.0, fw_dt = 0.0;
  // theta-method: U^{n-1}, the (1 - theta)-weighted level-n spatial vector and the
  // nodal (phi^n - phi^{n-1})/dt of the Eq. (theta) estimate
  double *Unm1 = nullptr, *Fold = nullptr, *phold = nullptr;
  bool old_valid = false;
  // weights of the solid fraction S = w^T U + |Omega|/2 (filled on first use)
  double* sfw = nullptr;
};

namespace {


int fail(tusas_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define TCK(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(h, TUSAS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

// Start / stop a timed region of class `cls` on the handle's stream.
size_t tbeg(tusas_handle* h) {
  if (!h->timers_on) return (size_t)-1;
  while (h->ev.size() < h->ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
    h->ev.push_back(e);
  }
  const size_t i = h->ev_used;
  h->ev_used += 2;
  cudaEventRecord(h->ev[i], h->st);
  return i;
}
void tend(tusas_handle* h, int cls, size_t i) {
  if (i == (size_t)-1) return;
  cudaEventRecord(h->ev[i + 1], h->st);
  h->marks.push_back(std::make_pair(cls, i));
}
// Fold recorded event pairs into the per-class sums (stream must be idle).
void tcollect(tusas_handle* h) {
  for (auto& mk : h->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[mk.second], h->ev[mk.second + 1]) == cudaSuccess) {
      h->t_ms[mk.first] += ms;
      h->t_cnt[mk.first] += 1;
    }
  }
  h->marks.clear();
  h->ev_used = 0;
}

int validate(const tusas_mesh* m, const tusas_params* p, std::string& why) {
  if (!m || !p) {
    why = "null mesh or params";
    return TUSAS_EINVAL;
  }
  if (m->dim != 2 && m->dim != 3) {
    why = "dim must be 2 or 3";
    return TUSAS_EINVAL;
  }
  if (m->nx < 1 || m->ny < 1 || (m->dim == 3 && m->nz < 1) || (m->dim == 2 && m->nz != 0)) {
    why = "element counts must be >= 1 (nz = 0 in 2D)";
    return TUSAS_EINVAL;
  }
  if (!(m->h > 0.0) || !isfinite(m->h)) {
    why = "h must be positive and finite";
    return TUSAS_EINVAL;
  }
  if (m->order < 0 || m->order > 2) {
    why = "order must be 0 or 1 (Q1) or 2 (Q2)";
    return TUSAS_EINVAL;
  }
  const int po = m->order == 2 ? 2 : 1;
  const double nodes = (double)(po * m->nx + 1) * (po * m->ny + 1) * (m->dim == 3 ? po * m->nz + 1 : 1);
  if (nodes > 2.0e9) {
    why = "mesh too large (more than 2e9 nodes)";
    return TUSAS_EINVAL;
  }
  if (p->model != 0 && p->model != 1) {
    why = "model must be 0 (pure metal) or 1 (alloy)";
    return TUSAS_EINVAL;
  }
  if (p->model == 0 && p->k != 1.0) {
    why = "the pure-metal model needs k = 1";
    return TUSAS_EINVAL;
  }
  if (!(p->theta >= 0.0 && p->theta <= 1.0) || (p->phihat_form != 0 && p->phihat_form != 1)) {
    why = "theta must be in [0, 1], phihat_form 0 or 1";
    return TUSAS_EINVAL;
  }
  if (!(p->W0 > 0) || !(p->tau0 > 0) || !(p->D >= 0) || !(p->eps4 >= 0 && p->eps4 < 0.25)) {
    why = "W0, tau0 must be > 0, D >= 0, 0 <= eps4 < 1/4";
    return TUSAS_EINVAL;
  }
  if (p->model == 1 && p->lT != 0.0 && !isfinite(p->lT)) {
    why = "lT must be finite";
    return TUSAS_EINVAL;
  }
  if (p->precond < 0 || p->precond > 2 || p->jvp_mode < 0 || p->jvp_mode > 1 || p->time_form < 0 ||
      p->time_form > 1) {
    why = "precond in 0..2, jvp_mode in 0..1, time_form in 0..1";
    return TUSAS_EINVAL;
  }
  if (p->gmres_restart < 1 || p->gmres_restart > 30 || p->gmres_maxit < 1 || p->newton_maxit < 0 ||
      p->newton_maxit > 30 || p->linesearch_max < 0) {
    why = "gmres_restart in 1..30, gmres_maxit >= 1, newton_maxit in 0..30, linesearch_max >= 0";
    return TUSAS_EINVAL;
  }
  if (p->precond == 2 && (p->mg_levels < 1 || p->cheb_degree < 1 || p->coarse_degree < 1)) {
    why = "mg_levels, cheb_degree, coarse_degree must be >= 1";
    return TUSAS_EINVAL;
  }
  return TUSAS_OK;
}

void fill_phys(tusas_handle* h) {
  tusas::DevPhys P;
  const tusas_params& p = h->prm;
  P.model = p.model;
  P.time_form = p.time_form;
  P.jat_norm = p.jat_normalised;
  P.W0 = p.W0;
  P.tau0 = p.tau0;
  P.eps4 = p.eps4;
  P.lam = p.lam;
  P.D = p.D;
  P.k = p.k;
  P.lT = p.lT;
  P.Vp = p.Vp;
  P.zT = p.zT;
  P.dt = h->dt;
  P.idt = h->dt > 0 ? 1.0 / h->dt : 0.0;
  P.t_new = h->t + h->dt;
  P.has_g4 = p.model == 1 && p.lT != 0.0;
  P.theta = p.theta;
  P.thW2 = p.theta * p.W0 * p.W0;
  P.thD = p.theta * p.D;
  P.phihat_old = (p.theta != 1.0 && p.phihat_form == 0) ? 1 : 0;
  P.dphat = P.phihat_old ? p.theta * P.idt : P.idt;
  tusas::elem_ctx_init(h->ec, h->dm, P);
  h->old_valid = false;
}

// Level-n quantities of the theta-method for the current state (once per state / dt).
int ensure_old(tusas_handle* h) {
  if (h->prm.theta == 1.0 || h->old_valid) return TUSAS_OK;
  TCK(tusas::elem_run(tusas::M_OLD, h->ec, h->Un, h->Un, nullptr, h->Fold, nullptr, h->st));
  if (h->ec.P.phihat_old) {
    TCK(tusas::vxpay(h->nn, h->Un, -1.0, nullptr, h->Unm1, h->phold, h->st));
    TCK(tusas::vscal(h->nn, h->ec.P.idt, h->phold, h->st));
  }
  h->old_valid = true;
  return TUSAS_OK;
}

const double* old_init(tusas_handle* h) { return h->prm.theta == 1.0 ? nullptr : h->Fold; }
const double* old_ph(tusas_handle* h) { return h->ec.P.phihat_old ? h->phold : nullptr; }

int ensure_lin(tusas_handle* h, bool trial) {
  if (!h->lin) {
    h->lin_n = tusas::elem_lin_doubles(h->ec);
    if (tusas::dev_malloc(&h->lin, sizeof(double) * h->lin_n) != cudaSuccess)
      return fail(h, TUSAS_ENOMEM, "linearisation store allocation");
  }
  if (trial && !h->lin_t && tusas::dev_malloc(&h->lin_t, sizeof(double) * h->lin_n) != cudaSuccess)
    return fail(h, TUSAS_ENOMEM, "trial linearisation store allocation");
  return TUSAS_OK;
}

int ready(tusas_handle* h) {
  if (!h) return TUSAS_EINVAL;
  if (!h->have_state || !(h->dt > 0)) return fail(h, TUSAS_EINVAL, "call tusas_set_state with dt > 0 first");
  return TUSAS_OK;
}

// ||x||^2 into device scalar slot `slot` (no synchronisation)
cudaError_t norm2_dev(tusas_handle* h, const double* x, int slot) {
  return tusas::multidot(h->N, 1, x, 0, x, h->partials, h->sc + slot, h->st);
}

int host_norm(tusas_handle* h, const double* x, double* out) {
  TCK(norm2_dev(h, x, 200));
  double v;
  TCK(cudaMemcpyAsync(&v, h->sc + 200, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  TCK(cudaStreamSynchronize(h->st));
  *out = sqrt(v);
  return TUSAS_OK;
}

__global__ void k_fd_eps(const double* unorm2, const double* vnorm2, double* eps_out) {
  const double un = sqrt(*unorm2), vn = sqrt(*vnorm2);
  if (vn == 0.0) {
    eps_out[0] = 0.0;
    eps_out[1] = 0.0;
  } else {
    const double e = sqrt((1.0 + un) * 2.220446049250313e-16) / vn;
    eps_out[0] = e;
    eps_out[1] = 1.0 / e;
  }
}

// Jv = (F(U + eps v) - F0)/eps with ||U||^2 already in sc[210]
int fd_jv(tusas_handle* h, const double* U, const double* F0, const double* v, double* Jv) {
  TCK(norm2_dev(h, v, 211));
  k_fd_eps<<<1, 1, 0, h->st>>>(h->sc + 210, h->sc + 211, h->sc + 212);
  tusas::count_launches(1);
  TCK(tusas::vxpay(h->N, U, 0.0, h->sc + 212, v, h->tmp2, h->st));
  TCK(tusas::elem_run(tusas::M_RES, h->ec, h->tmp2, h->Un, nullptr, Jv, nullptr, h->st, old_init(h), old_ph(h)));
  TCK(tusas::vfdq(h->N, F0, Jv, h->sc + 213, h->st));
  return TUSAS_OK;
}

}  // namespace

extern "C" {

int tusas_create(const tusas_mesh* mesh, const tusas_params* params, tusas_handle** out) {
  if (!out) return TUSAS_EINVAL;
  *out = nullptr;
  std::string why;
  int rc = validate(mesh, params, why);
  if (rc) return rc;
  {
    // admission against the device-bytes cap before any CUDA call: the vectors and the Krylov basis
    const int po = mesh->order == 2 ? 2 : 1;
    const long long nn = (long long)(po * mesh->nx + 1) * (po * mesh->ny + 1) * (mesh->dim == 3 ? po * mesh->nz + 1 : 1);
    const long long base = (long long)sizeof(double) * 2 * nn * (11 + 2 * params->gmres_restart + 1);
    if (!tusas::dev_bytes_admit(base)) return TUSAS_ENOMEM;
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return TUSAS_ECUDA;
  tusas_handle* h = new tusas_handle();
  h->mesh = *mesh;
  h->prm = *params;
  h->device = device;
  tusas::DevMesh& d = h->dm;
  d.dim = mesh->dim;
  d.order = mesh->order == 2 ? 2 : 1;
  d.nx = mesh->nx;
  d.ny = mesh->ny;
  d.nz = mesh->dim == 3 ? mesh->nz : 0;
  d.nnx = d.order * mesh->nx + 1;
  d.nny = d.order * mesh->ny + 1;
  d.nnz = mesh->dim == 3 ? d.order * mesh->nz + 1 : 1;
  d.nn = (i64)d.nnx * d.nny * d.nnz;
  d.ne = (i64)d.nx * d.ny * (mesh->dim == 3 ? d.nz : 1);
  d.h = mesh->h;
  d.x0 = mesh->x0;
  d.y0 = mesh->y0;
  d.z0 = mesh->z0;
  h->nn = d.nn;
  h->N = 2 * d.nn;
  fill_phys(h);
  double** vecs[] = {&h->Un, &h->U, &h->F, &h->Ft, &h->dU, &h->Ut, &h->tmp, &h->tmp2, &h->Unm1, &h->Fold, &h->phold};
  for (double** v : vecs) {
    cudaError_t e = tusas::dev_malloc(v, sizeof(double) * h->N);
    if (e != cudaSuccess) {
      tusas_destroy(h);
      return TUSAS_ENOMEM;
    }
  }
  h->m = params->gmres_restart;
  if (tusas::dev_malloc(&h->V, sizeof(double) * h->N * (h->m + 1)) != cudaSuccess ||
      tusas::dev_malloc(&h->Z, sizeof(double) * h->N * h->m) != cudaSuccess ||
      tusas::dev_malloc(&h->partials, sizeof(double) * std::max(tusas::reduce_blocks(), tusas::gs_blocks()) * 32) !=
          cudaSuccess ||
      tusas::dev_malloc(&h->sc, sizeof(double) * 256) != cudaSuccess ||
      tusas::dev_malloc(&h->hess, sizeof(double) * ((h->m + 1) * h->m + 3 * h->m + 8)) != cudaSuccess) {
    tusas_destroy(h);
    return TUSAS_ENOMEM;
  }
  if (cudaHostAlloc(&h->st_host, sizeof(double) * 4, cudaHostAllocMapped) != cudaSuccess) {
    h->st_host = nullptr;
    tusas_destroy(h);
    return TUSAS_ENOMEM;
  }
  if (cudaHostGetDevicePointer(&h->st_host_dev, h->st_host, 0) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_st, cudaEventDisableTiming) != cudaSuccess) {
    h->ev_st = nullptr;
    tusas_destroy(h);
    return TUSAS_ECUDA;
  }
  if (params->precond > 0) {
    cudaError_t e = h->pc.create(h->dm, params->precond, params->smoother_fp32, params->mg_levels,
                                 params->cheb_degree, params->coarse_degree);
    if (e != cudaSuccess) {
      tusas_destroy(h);
      return e == cudaErrorMemoryAllocation ? TUSAS_ENOMEM : TUSAS_ECUDA;
    }
  }
  *out = h;
  return TUSAS_OK;
}

void tusas_destroy(tusas_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  cudaDeviceSynchronize();
  double* vecs[] = {h->Un, h->U, h->F, h->Ft, h->dU, h->Ut, h->tmp, h->tmp2, h->lin, h->lin_t, h->V, h->Z,
                    h->partials, h->sc, h->hess, h->Unm1, h->Fold, h->phold};
  for (double* v : vecs) tusas::dev_free(v);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  for (double* p : h->ckpt) tusas::dev_free(p);
  for (double* p : h->seg) tusas::dev_free(p);
  tusas::dev_free(h->lam);
  tusas::dev_free(h->lam_rhs);
  tusas::dev_free(h->Ufinal);
  tusas::dev_free(h->sfw);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->ev_st) cudaEventDestroy(h->ev_st);
  h->pc.destroy();
  delete h;
}

int tusas_set_stream(tusas_handle* h, void* s) {
  if (!h) return TUSAS_EINVAL;
  h->st = (cudaStream_t)s;
  return TUSAS_OK;
}

int tusas_set_params(tusas_handle* h, const tusas_params* p) {
  if (!h) return TUSAS_EINVAL;
  std::string why;
  int rc = validate(&h->mesh, p, why);
  if (rc) return fail(h, rc, why);
  if (p->gmres_restart > h->m || p->precond != h->prm.precond || p->smoother_fp32 != h->prm.smoother_fp32 ||
      p->mg_levels != h->prm.mg_levels || p->model != h->prm.model)
    return fail(h, TUSAS_EINVAL, "restart length, preconditioner kind/precision/levels and model are fixed at create");
  h->prm = *p;
  h->pc.cheb_degree = p->cheb_degree;
  h->pc.coarse_degree = p->coarse_degree;
  fill_phys(h);
  h->pc_ready = false;
  return TUSAS_OK;
}

long long tusas_ndofs(const tusas_handle* h) { return h ? (long long)h->N : -1; }

double tusas_time(const tusas_handle* h) { return h ? h->t : 0.0; }

int tusas_set_state(tusas_handle* h, const double* U, double t, double dt) {
  if (!h || !U) return TUSAS_EINVAL;
  if (!(dt > 0) || !isfinite(dt) || !isfinite(t)) return fail(h, TUSAS_EINVAL, "dt must be positive, t finite");
  TCK(cudaMemcpyAsync(h->Un, U, sizeof(double) * h->N, cudaMemcpyDefault, h->st));
  TCK(cudaMemcpyAsync(h->Unm1, h->Un, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
  TCK(cudaStreamSynchronize(h->st));
  h->t = t;
  h->dt = dt;
  h->have_state = true;
  h->pc_ready = false;
  fill_phys(h);
  return TUSAS_OK;
}

int tusas_set_history(tusas_handle* h, const double* Unm1) {
  int rc = ready(h);
  if (rc) return rc;
  if (!Unm1) return fail(h, TUSAS_EINVAL, "null vector");
  TCK(cudaMemcpyAsync(h->Unm1, Unm1, sizeof(double) * h->N, cudaMemcpyDefault, h->st));
  TCK(cudaStreamSynchronize(h->st));
  h->old_valid = false;
  return TUSAS_OK;
}

int tusas_get_state(tusas_handle* h, double* U) {
  if (!h || !U) return TUSAS_EINVAL;
  if (!h->have_state) return fail(h, TUSAS_EINVAL, "no state set");
  TCK(cudaMemcpyAsync(U, h->Un, sizeof(double) * h->N, cudaMemcpyDefault, h->st));
  TCK(cudaStreamSynchronize(h->st));
  return TUSAS_OK;
}

int tusas_residual(tusas_handle* h, const double* U, double* F) {
  int rc = ready(h);
  if (rc) return rc;
  if (!U || !F || U == F) return fail(h, TUSAS_EINVAL, "null or aliased vectors");
  if ((rc = ensure_old(h))) return rc;
  const size_t t0 = tbeg(h);
  TCK(tusas::elem_run(tusas::M_RES, h->ec, U, h->Un, nullptr, F, nullptr, h->st, old_init(h), old_ph(h)));
  tend(h, TUSAS_T_RESIDUAL, t0);
  return TUSAS_OK;
}

int tusas_jvp(tusas_handle* h, const double* U, const double* v, double* Jv) {
  int rc = ready(h);
  if (rc) return rc;
  if (!U || !v || !Jv || Jv == U || Jv == v) return fail(h, TUSAS_EINVAL, "null or aliased vectors");
  rc = ensure_lin(h, false);
  if (rc) return rc;
  if ((rc = ensure_old(h))) return rc;
  size_t t0 = tbeg(h);
  TCK(tusas::elem_run(tusas::M_RES_LIN, h->ec, U, h->Un, nullptr, h->tmp, h->lin, h->st, old_init(h), old_ph(h)));
  tend(h, TUSAS_T_RESIDUAL_LIN, t0);
  t0 = tbeg(h);
  TCK(tusas::elem_run(tusas::M_JV, h->ec, nullptr, nullptr, v, Jv, h->lin, h->st));
  tend(h, TUSAS_T_JV, t0);
  return TUSAS_OK;
}

int tusas_jvp_fd(tusas_handle* h, const double* U, const double* v, double* Jv) {
  int rc = ready(h);
  if (rc) return rc;
  if (!U || !v || !Jv || Jv == U || Jv == v) return fail(h, TUSAS_EINVAL, "null or aliased vectors");
  if ((rc = ensure_old(h))) return rc;
  TCK(tusas::elem_run(tusas::M_RES, h->ec, U, h->Un, nullptr, h->tmp, nullptr, h->st, old_init(h), old_ph(h)));
  TCK(norm2_dev(h, U, 210));
  return fd_jv(h, U, h->tmp, v, Jv);
}

int tusas_jtvp(tusas_handle* h, const double* U, const double* w, double* JTw) {
  int rc = ready(h);
  if (rc) return rc;
  if (!U || !w || !JTw || JTw == U || JTw == w) return fail(h, TUSAS_EINVAL, "null or aliased vectors");
  rc = ensure_lin(h, false);
  if (rc) return rc;
  if ((rc = ensure_old(h))) return rc;
  size_t t0 = tbeg(h);
  TCK(tusas::elem_run(tusas::M_RES_LIN, h->ec, U, h->Un, nullptr, h->tmp, h->lin, h->st, old_init(h), old_ph(h)));
  tend(h, TUSAS_T_RESIDUAL_LIN, t0);
  t0 = tbeg(h);
  TCK(tusas::elem_run(tusas::M_JTV, h->ec, nullptr, nullptr, w, JTw, h->lin, h->st));
  tend(h, TUSAS_T_ADJOINT, t0);
  return TUSAS_OK;
}

int tusas_jtvp_prev(tusas_handle* h, const double* U, const double* w, double* out) {
  int rc = ready(h);
  if (rc) return rc;
  if (!U || !w || !out || out == U || out == w) return fail(h, TUSAS_EINVAL, "null or aliased vectors");
  if (h->ec.P.phihat_old) return fail(h, TUSAS_EINVAL, "(dF/dU^n)^T w needs phihat_form 1 when theta < 1");
  const size_t t0 = tbeg(h);
  TCK(tusas::elem_run(tusas::M_PREV_T, h->ec, U, h->Un, w, out, nullptr, h->st));
  tend(h, TUSAS_T_ADJOINT, t0);
  return TUSAS_OK;
}

int tusas_dFdp(tusas_handle* h, const double* U, int which, double* dF) {
  int rc = ready(h);
  if (rc) return rc;
  if (!U || !dF || U == dF) return fail(h, TUSAS_EINVAL, "null or aliased vectors");
  if (which != 0) return fail(h, TUSAS_EINVAL, "only which = 0 (eps4) is available");
  if (h->ec.P.phihat_old) return fail(h, TUSAS_EINVAL, "dF/dp needs phihat_form 1 when theta < 1");
  const size_t t0 = tbeg(h);
  TCK(tusas::elem_run(tusas::M_DEPS, h->ec, U, h->Un, nullptr, dF, nullptr, h->st));
  tend(h, TUSAS_T_ADJOINT, t0);
  return TUSAS_OK;
}

int tusas_precond_setup(tusas_handle* h, const double* U) {
  int rc = ready(h);
  if (rc) return rc;
  if (!U) return fail(h, TUSAS_EINVAL, "null vector");
  const size_t t0 = tbeg(h);
  TCK(h->pc.setup(h->ec, h->prm.theta, U, h->Un, h->st));
  tend(h, TUSAS_T_PC_SETUP, t0);
  h->pc_ready = true;
  return TUSAS_OK;
}

int tusas_precond_apply(tusas_handle* h, const double* r, double* z) {
  if (!h || !r || !z || r == z) return fail(h, TUSAS_EINVAL, "null or aliased vectors");
  if (h->prm.precond == 0) {
    TCK(tusas::vcopy(h->N, r, z, h->st));
    return TUSAS_OK;
  }
  if (!h->pc_ready) return fail(h, TUSAS_EINVAL, "call tusas_precond_setup first");
  h->pc_input_for = nullptr;
  const size_t t0 = tbeg(h);
  TCK(h->pc.apply(r, z, h->st));
  tend(h, TUSAS_T_PC_APPLY, t0);
  return TUSAS_OK;
}

int tusas_dot(tusas_handle* h, const double* x, const double* y, long long n, double* result) {
  if (!h || !x || !y || !result || n < 0) return TUSAS_EINVAL;
  if (n == 0) {
    *result = 0.0;
    return TUSAS_OK;
  }
  TCK(tusas::multidot(n, 1, x, 0, y, h->partials, h->sc + 200, h->st));
  TCK(cudaMemcpyAsync(result, h->sc + 200, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  TCK(cudaStreamSynchronize(h->st));
  return TUSAS_OK;
}

int tusas_timers(tusas_handle* h, int enable) {
  if (!h) return TUSAS_EINVAL;
  TCK(cudaStreamSynchronize(h->st));
  h->marks.clear();
  h->ev_used = 0;
  for (int i = 0; i < TUSAS_NTIMERS; ++i) {
    h->t_ms[i] = 0.0;
    h->t_cnt[i] = 0;
  }
  h->timers_on = enable != 0;
  return TUSAS_OK;
}

int tusas_get_timers(tusas_handle* h, double* ms, long long* counts) {
  if (!h || !ms || !counts) return TUSAS_EINVAL;
  TCK(cudaStreamSynchronize(h->st));
  tcollect(h);
  for (int i = 0; i < TUSAS_NTIMERS; ++i) {
    ms[i] = h->t_ms[i];
    counts[i] = h->t_cnt[i];
  }
  return TUSAS_OK;
}

const char* tusas_last_error(const tusas_handle* h) {
  if (!h) return "null handle";
  return h->err.empty() ? "no error" : h->err.c_str();
}

// ---------------------------------------------------------------------------
// Newton-Krylov step
// ---------------------------------------------------------------------------

// Krylov operators: exact tangent (stored linearisation), finite difference, transposed tangent.
enum { OP_EXACT = 0, OP_FD = 1, OP_TRANS = 2 };

static int jv_apply(tusas_handle* h, int op, const double* z, double* out) {
  const size_t t0 = tbeg(h);
  if (op == OP_EXACT) {
    TCK(tusas::elem_run(tusas::M_JV, h->ec, nullptr, nullptr, z, out, h->lin, h->st));
  } else if (op == OP_TRANS) {
    TCK(tusas::elem_run(tusas::M_JTV, h->ec, nullptr, nullptr, z, out, h->lin, h->st));
  } else {
    int rc = fd_jv(h, h->U, h->F, z, out);
    if (rc) return rc;
  }
  tend(h, op == OP_TRANS ? TUSAS_T_ADJOINT : TUSAS_T_JV, t0);
  return TUSAS_OK;
}

static int prec_apply(tusas_handle* h, const double* r, double* z) {
  if (h->prm.precond == 0) {
    TCK(tusas::vcopy(h->N, r, z, h->st));
    return TUSAS_OK;
  }
  const bool input_ready = r == h->pc_input_for;
  h->pc_input_for = nullptr;
  const size_t t0 = tbeg(h);
  TCK(h->pc.apply(r, z, h->st, input_ready));
  tend(h, TUSAS_T_PC_APPLY, t0);
  return TUSAS_OK;
}

// New column j of the Arnoldi relation and its Givens rotation, on the device. One block
// of 32 (j + 2) threads: warp c reduces column c of the second Gram-Schmidt pass's block
// partial sums (c <= j: h2[c] = V_c . w1, c = j + 1: ||w1||^2), in the order of the
// deterministic reductions; then one thread forms H[i][j] = h1[i] + h2[i] and
// H[j+1][j] = ||w2||, w2 = w1 - V h2, from the Pythagorean identity
// ||w2||^2 = ||w1||^2 - ||h2||^2 (exact for an orthonormal V; the classical Gram-Schmidt
// variant with the Pythagorean norm, Smoktunowicz, Barlow and Langou, Numer. Math. 105
// (2006)); h2 is the reorthogonalisation correction, of the order of the rounding of the
// first pass, so the difference loses no digits unless w lies in span(V) to machine
// precision, where H[j+1][j] and the GMRES residual vanish to rounding and the cycle ends.
// The earlier rotations are applied to the column, the new one formed from its last two
// entries, g updated. st[0] = |g[j+1]| (the residual estimate), st[1] = ||w2||,
// st[2] = 1/||w2|| (0 if ||w2|| = 0; the last pass scales w2 by it), st[3] = the new
// diagonal entry, copied to st_host (mapped pinned memory) as well.
__global__ void k_arnoldi_givens(int j, int m, int nb, const double* __restrict__ partials,
                                 const double* __restrict__ h1, double* __restrict__ h2, double* __restrict__ H,
                                 double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                                 double* __restrict__ st, double* __restrict__ st_host) {
  __shared__ double red[32];
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c <= j + 1) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += partials[b * (i64)32 + c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) red[c] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double q = red[j + 1];
  for (int i = 0; i <= j; ++i) {
    const double c2 = red[i];
    h2[i] = c2;
    q = fma(-c2, c2, q);
    H[i * m + j] = h1[i] + c2;
  }
  const double hn = sqrt(q > 0.0 ? q : 0.0);
  H[(j + 1) * m + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * m + j], bb = H[(i + 1) * m + j];
    H[i * m + j] = cs[i] * a + sn[i] * bb;
    H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
  }
  const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
  cs[j] = H[j * m + j] / den;
  sn[j] = H[(j + 1) * m + j] / den;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  const double o[4] = {fabs(g[j + 1]), hn, hn > 0.0 ? 1.0 / hn : 0.0, den};
  for (int i = 0; i < 4; ++i) st[i] = st_host[i] = o[i];
}

// g = (beta, 0, ..., 0) at the start of a cycle
__global__ void k_givens_start(int m, double beta, double* __restrict__ g) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = i == 0 ? beta : 0.0;
}

// Flexible right-preconditioned restarted GMRES with classical Gram-Schmidt
// applied twice, x0 = 0; solves J x = b (b = -F) to ||b - J x|| <= tol_abs.
// resid_out: the final residual norm (the Givens estimate, or the true norm after a restart).
static int gmres(tusas_handle* h, int op, const double* b, double* x, double tol_abs, int* its_out,
                 tusas_stats* stats, bool* converged = nullptr, int maxit = -1, double* resid_out = nullptr) {
  const int m = h->prm.gmres_restart;
  const i64 N = h->N;
  // device Hessenberg, rotations, g and status (k_arnoldi_givens), sized for the allocated restart
  double* dH = h->hess;
  double* dcs = dH + (h->m + 1) * h->m;
  double* dsn = dcs + h->m;
  double* dg = dsn + h->m;
  double* dst = dg + h->m + 1;
  std::vector<double> H((m + 1) * m), g(m + 1), y(m);
  double stat[4];
  TCK(cudaMemsetAsync(x, 0, sizeof(double) * N, h->st));
  h->pc_input_for = nullptr;
  int its = 0;
  // r = b
  double* r = h->V;  // V_0 doubles as the residual buffer
  TCK(tusas::vcopy(N, b, r, h->st));
  double beta;
  int rc = host_norm(h, r, &beta);
  if (rc) return rc;
  double resid = beta;
  if (maxit < 0) maxit = h->prm.gmres_maxit;
  while (beta > tol_abs && its < maxit) {
    if (!isfinite(beta)) return fail(h, TUSAS_ENONFINITE, "non-finite GMRES residual");
    TCK(tusas::vscal(N, 1.0 / beta, r, h->st));  // V_0 = r / beta
    k_givens_start<<<1, 32, 0, h->st>>>(m, beta, dg);
    tusas::count_launches(1);
    int mu = 0;
    for (int j = 0; j < m; ++j) {
      double* Vj = h->V + (i64)j * N;
      double* Zj = h->Z + (i64)j * N;
      double* w = h->V + (i64)(j + 1) * N;
      rc = prec_apply(h, Vj, Zj);
      if (rc) return rc;
      rc = jv_apply(h, op, Zj, w);
      if (rc) return rc;
      if (stats) stats->jv_evals++;
      ++its;
      // classical Gram-Schmidt applied twice (CGS2) in three passes over the basis: h = V^T w;
      // w -= V h fused with h2 = V^T w and ||w||^2; w = (w - V h2) / ||w - V h2|| with the norm
      // from the Pythagorean identity (k_arnoldi_givens, between the last two passes)
      const size_t to = tbeg(h);
      TCK(tusas::gs_pass(0, N, j + 1, h->V, N, nullptr, nullptr, w, h->partials, h->sc, h->st));
      TCK(tusas::gs_pass(1, N, j + 1, h->V, N, h->sc, nullptr, w, h->partials, nullptr, h->st));
      k_arnoldi_givens<<<1, 32 * (j + 2), 0, h->st>>>(j, m, tusas::gs_blocks(), h->partials, h->sc, h->sc + 64, dH,
                                                        dcs, dsn, dg, dst, h->st_host_dev);
      tusas::count_launches(1);
      TCK(cudaGetLastError());
      TCK(cudaEventRecord(h->ev_st, h->st));
      // the FP32 multigrid's input for w, preconditioned next unless the cycle ends here
      tusas::GsNarrow nw;
      const bool narrow_w = j + 1 < m && h->prm.precond != 0 && h->pc.fp32_input(&nw.b, &nw.db, &nw.dinv);
      TCK(tusas::gs_pass(2, N, j + 1, h->V, N, h->sc + 64, dst + 2, w, h->partials, nullptr, h->st,
                         narrow_w ? nw : tusas::GsNarrow()));
      h->pc_input_for = narrow_w ? w : nullptr;
      tend(h, TUSAS_T_ORTHO, to);
      // the status is read while the last pass runs
      TCK(cudaEventSynchronize(h->ev_st));
      for (int i = 0; i < 4; ++i) stat[i] = ((volatile double*)h->st_host)[i];
      if (!isfinite(stat[1]) || !isfinite(stat[0])) return fail(h, TUSAS_ENONFINITE, "non-finite Krylov vector");
      resid = stat[0];
      mu = j + 1;
      if (resid <= tol_abs || its >= maxit || stat[3] == 0.0) break;
    }
    h->pc_input_for = nullptr;
    // the triangle R = H[0..mu-1][0..mu-1] and g once per cycle
    TCK(cudaMemcpyAsync(H.data(), dH, sizeof(double) * mu * m, cudaMemcpyDeviceToHost, h->st));
    TCK(cudaMemcpyAsync(g.data(), dg, sizeof(double) * (mu + 1), cudaMemcpyDeviceToHost, h->st));
    TCK(cudaStreamSynchronize(h->st));
    for (int i = mu - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < mu; ++k) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    TCK(cudaMemcpyAsync(h->sc + 128, y.data(), sizeof(double) * mu, cudaMemcpyHostToDevice, h->st));
    TCK(tusas::multi_comb(N, mu, h->Z, N, h->sc + 128, x, h->st));
    if (resid <= tol_abs || its >= maxit) break;
    // restart: r = b - J x
    rc = jv_apply(h, op, x, h->tmp);
    if (rc) return rc;
    if (stats) stats->jv_evals++;
    TCK(tusas::vcopy(N, b, r, h->st));
    TCK(tusas::vaxpy(N, -1.0, h->tmp, r, h->st));
    rc = host_norm(h, r, &beta);
    if (rc) return rc;
    resid = beta;
  }
  *its_out = its;
  if (converged) *converged = resid <= tol_abs;
  if (resid_out) *resid_out = resid;
  return TUSAS_OK;
}

static double forcing(const tusas_params& p, int l, double fn, double fprev, double eta_prev) {
  if (l == 0) return p.eta0;
  double eta = p.gamma * pow(fn / fprev, p.omega);
  eta = std::max(eta, std::max(p.gamma * pow(eta_prev, p.omega), p.eta_min));
  return std::min(p.eta_max, eta);
}

int tusas_step(tusas_handle* h, tusas_stats* stats) {
  int rc = ready(h);
  if (rc) return rc;
  tusas_stats S = {};
  const tusas_params& p = h->prm;
  const bool exact = p.jvp_mode == 1;
  const i64 N = h->N;
  if (exact) {
    rc = ensure_lin(h, true);
    if (rc) return rc;
  }
  TCK(tusas::vcopy(N, h->Un, h->U, h->st));
  if ((rc = ensure_old(h))) return rc;
  size_t t0 = tbeg(h);
  TCK(tusas::elem_run(exact ? tusas::M_RES_LIN : tusas::M_RES, h->ec, h->U, h->Un, nullptr, h->F, h->lin, h->st,
                      old_init(h), old_ph(h)));
  tend(h, exact ? TUSAS_T_RESIDUAL_LIN : TUSAS_T_RESIDUAL, t0);
  S.residual_evals = 1;
  double fn;
  rc = host_norm(h, h->F, &fn);
  if (rc) return rc;
  if (!isfinite(fn)) return fail(h, TUSAS_ENONFINITE, "non-finite initial residual norm");
  S.fnorm0 = S.fnorm = fn;
  const double tol = p.newton_rtol * fn + p.newton_atol;
  double eta_prev = p.eta0, fprev = 0.0;
  bool converged = false;
  for (int l = 0; l <= p.newton_maxit; ++l) {
    if (S.fnorm < tol || S.fnorm == 0.0) {
      converged = true;
      break;
    }
    if (l == p.newton_maxit) break;
    const double eta = forcing(p, l, S.fnorm, fprev, eta_prev);
    if (p.precond > 0) {
      t0 = tbeg(h);
      TCK(h->pc.setup(h->ec, p.theta, h->U, h->Un, h->st));
      tend(h, TUSAS_T_PC_SETUP, t0);
      h->pc_ready = true;
    }
    if (!exact) TCK(norm2_dev(h, h->U, 210));
    // b = -F (in Ft), solve J dU = b
    TCK(tusas::vfill(N, 0.0, h->Ft, h->st));
    TCK(tusas::vaxpy(N, -1.0, h->F, h->Ft, h->st));
    int its = 0;
    double rlin = 0.0;
    rc = gmres(h, exact ? OP_EXACT : OP_FD, h->Ft, h->dU, eta * S.fnorm, &its, &S, nullptr, -1, &rlin);
    if (rc) return rc;
    S.gmres_its += its;
    if (S.newton_its < 32) S.gmres_per_newton[S.newton_its] = its;
    double lam = 1.0, ftn = 0.0;
    bool accepted = false;
    for (int ls = 0; ls <= p.linesearch_max; ++ls) {
      TCK(tusas::vxpay(N, h->U, lam, nullptr, h->dU, h->Ut, h->st));
      // When the linear model ||F + J dU|| is below the Newton tolerance the full step is
      // expected to converge: evaluate F alone, and store the linearisation at the trial
      // point only if the Newton loop goes on.
      const bool lin_now = exact && !(ls == 0 && rlin <= tol);
      t0 = tbeg(h);
      TCK(tusas::elem_run(lin_now ? tusas::M_RES_LIN : tusas::M_RES, h->ec, h->Ut, h->Un, nullptr, h->Ft, h->lin_t,
                          h->st, old_init(h), old_ph(h)));
      tend(h, lin_now ? TUSAS_T_RESIDUAL_LIN : TUSAS_T_RESIDUAL, t0);
      S.residual_evals++;
      rc = host_norm(h, h->Ft, &ftn);
      if (rc) return rc;
      if (!isfinite(ftn)) return fail(h, TUSAS_ENONFINITE, "non-finite residual norm in the line search");
      if (ftn <= S.fnorm) {
        accepted = true;
        if (exact && !lin_now && !(ftn < tol || ftn == 0.0)) {  // mispredicted: linearise here
          t0 = tbeg(h);
          TCK(tusas::elem_run(tusas::M_RES_LIN, h->ec, h->Ut, h->Un, nullptr, h->Ft, h->lin_t, h->st, old_init(h),
                              old_ph(h)));
          tend(h, TUSAS_T_RESIDUAL_LIN, t0);
          S.residual_evals++;
          rc = host_norm(h, h->Ft, &ftn);
          if (rc) return rc;
          if (!isfinite(ftn)) return fail(h, TUSAS_ENONFINITE, "non-finite residual norm in the line search");
        }
        break;
      }
      lam *= 0.5;
      S.linesearch_halvings++;
    }
    if (!accepted) break;
    std::swap(h->U, h->Ut);
    std::swap(h->F, h->Ft);
    if (exact) std::swap(h->lin, h->lin_t);
    fprev = S.fnorm;
    eta_prev = eta;
    S.fnorm = ftn;
    S.newton_its++;
  }
  S.converged = converged ? 1 : 0;
  if (stats) *stats = S;
  if (h->timers_on) {
    TCK(cudaStreamSynchronize(h->st));
    tcollect(h);
  }
  if (!converged) return fail(h, TUSAS_ENOCONV, "Newton did not converge");
  TCK(tusas::vcopy(N, h->Un, h->Unm1, h->st));
  TCK(tusas::vcopy(N, h->U, h->Un, h->st));
  TCK(cudaStreamSynchronize(h->st));
  h->t += h->dt;
  fill_phys(h);
  h->pc_ready = false;
  return TUSAS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Discrete adjoint through N implicit steps (not in the paper)
// ---------------------------------------------------------------------------
namespace {
int grow(tusas_handle* h, std::vector<double*>& v, size_t n) {
  while (v.size() < n) {
    double* p = nullptr;
    if (tusas::dev_malloc(&p, sizeof(double) * h->N) != cudaSuccess) return fail(h, TUSAS_ENOMEM, "checkpoint allocation");
    v.push_back(p);
  }
  return TUSAS_OK;
}
int ensure_vec(tusas_handle* h, double** p) {
  if (!*p && tusas::dev_malloc(p, sizeof(double) * h->N) != cudaSuccess) return fail(h, TUSAS_ENOMEM, "vector allocation");
  return TUSAS_OK;
}
int set_state_dev(tusas_handle* h, const double* U, double t) {
  TCK(cudaMemcpyAsync(h->Un, U, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
  h->t = t;
  fill_phys(h);
  h->pc_ready = false;
  return TUSAS_OK;
}
}  // namespace

static const int kAdjointMaxit = 1000;

extern "C" int tusas_forward(tusas_handle* h, const double* U0, double t0, double dt, int nsteps, int ckpt_every,
                             tusas_stats* total) {
  if (!h || !U0 || nsteps < 1 || ckpt_every < 1) return fail(h, TUSAS_EINVAL, "bad forward arguments");
  if (h->prm.theta != 1.0 && h->prm.phihat_form == 0)
    return fail(h, TUSAS_EINVAL, "the discrete adjoint needs phihat_form 1 when theta < 1");
  int rc = tusas_set_state(h, U0, t0, dt);
  if (rc) return rc;
  const size_t nck = (size_t)(nsteps + ckpt_every - 1) / ckpt_every + 1;
  rc = grow(h, h->ckpt, nck);
  if (rc) return rc;
  tusas_stats T = {};
  T.converged = 1;
  TCK(cudaMemcpyAsync(h->ckpt[0], h->Un, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
  for (int n = 1; n <= nsteps; ++n) {
    tusas_stats S = {};
    rc = tusas_step(h, &S);
    T.newton_its += S.newton_its;
    T.gmres_its += S.gmres_its;
    T.residual_evals += S.residual_evals;
    T.jv_evals += S.jv_evals;
    T.linesearch_halvings += S.linesearch_halvings;
    if (n == 1) T.fnorm0 = S.fnorm0;
    T.fnorm = S.fnorm;
    if (rc) {
      T.converged = 0;
      if (total) *total = T;
      return rc;
    }
    if (n % ckpt_every == 0)
      TCK(cudaMemcpyAsync(h->ckpt[n / ckpt_every], h->Un, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
  }
  rc = ensure_vec(h, &h->Ufinal);
  if (rc) return rc;
  TCK(cudaMemcpyAsync(h->Ufinal, h->Un, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
  TCK(cudaStreamSynchronize(h->st));
  h->fw_steps = nsteps;
  h->fw_every = ckpt_every;
  h->fw_t0 = t0;
  h->fw_dt = dt;
  if (total) *total = T;
  return TUSAS_OK;
}

extern "C" int tusas_adjoint(tusas_handle* h, const double* w, const double* d0, double* grad_eps4, double* grad_dir,
                             double* g0, double adj_rtol, tusas_stats* stats) {
  if (!h || !w || !grad_eps4) return fail(h, TUSAS_EINVAL, "null argument");
  if (h->fw_steps < 1) return fail(h, TUSAS_EINVAL, "call tusas_forward first");
  if (h->prm.theta != 1.0 && h->prm.phihat_form == 0)
    return fail(h, TUSAS_EINVAL, "the discrete adjoint needs phihat_form 1 when theta < 1");
  if (!(adj_rtol > 0.0)) return fail(h, TUSAS_EINVAL, "adj_rtol must be positive");
  const int N = h->fw_steps, c = h->fw_every;
  const double t0 = h->fw_t0, dt = h->fw_dt;
  const i64 n2 = h->N;
  int rc = ensure_lin(h, false);
  if (rc) return rc;
  if ((rc = ensure_vec(h, &h->lam)) || (rc = ensure_vec(h, &h->lam_rhs))) return rc;
  rc = grow(h, h->seg, (size_t)c + 2);  // seg[0..c]: one segment; seg[c+1]: U_{n+1} at a segment end
  if (rc) return rc;
  tusas_stats S = {};
  S.converged = 1;
  double geps = 0.0;
  const int nseg = (N + c - 1) / c;
  for (int k = nseg - 1; k >= 0; --k) {
    // recompute U_{kc} .. U_{min((k+1)c, N)} from checkpoint k
    const int n0 = k * c, n1 = std::min((k + 1) * c, N);
    TCK(cudaMemcpyAsync(h->seg[0], h->ckpt[k], sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->st));
    for (int n = n0 + 1; n <= n1; ++n) {
      rc = set_state_dev(h, h->seg[n - 1 - n0], t0 + (n - 1) * dt);
      if (rc) return rc;
      tusas_stats fs;
      rc = tusas_step(h, &fs);
      if (rc) return rc;
      TCK(cudaMemcpyAsync(h->seg[n - n0], h->Un, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->st));
    }
    for (int n = n1; n > n0; --n) {
      const double* Un_ = h->seg[n - n0];
      const double* Uprev = h->seg[n - 1 - n0];
      // rhs_n = w (n = N) or -(dF_{n+1}/dU_n)^T lam_{n+1}
      if (n == N) {
        TCK(tusas::vcopy(n2, w, h->lam_rhs, h->st));
      } else {
        // state pair (U_{n+1}, U_n): U_{n+1} is seg[n+1-n0] or, at a segment end, the first state of the next segment
        const double* Unext = (n + 1 - n0 <= c) ? h->seg[n + 1 - n0] : h->seg[c + 1];
        rc = set_state_dev(h, Un_, t0 + n * dt);
        if (rc) return rc;
        const size_t ta = tbeg(h);
        TCK(tusas::elem_run(tusas::M_PREV_T, h->ec, Unext, h->Un, h->lam, h->lam_rhs, nullptr, h->st));
        tend(h, TUSAS_T_ADJOINT, ta);
        TCK(tusas::vscal(n2, -1.0, h->lam_rhs, h->st));
      }
      // J_n^T lam_n = rhs_n at (U_n, U_{n-1})
      rc = set_state_dev(h, Uprev, t0 + (n - 1) * dt);
      if (rc) return rc;
      size_t ta = tbeg(h);
      TCK(tusas::elem_run(tusas::M_RES_LIN, h->ec, Un_, h->Un, nullptr, h->tmp, h->lin, h->st));
      tend(h, TUSAS_T_RESIDUAL_LIN, ta);
      if (h->prm.precond > 0) {
        ta = tbeg(h);
        TCK(h->pc.setup(h->ec, h->prm.theta, Un_, h->Un, h->st));
        tend(h, TUSAS_T_PC_SETUP, ta);
        h->pc_ready = true;
      }
      double bn;
      rc = host_norm(h, h->lam_rhs, &bn);
      if (rc) return rc;
      int its = 0;
      bool ok = true;
      // the adjoint solves must reach their tolerance: at least 1000 iterations whatever the
      // (possibly truncating) Newton-Krylov cap of the forward steps
      rc = gmres(h, OP_TRANS, h->lam_rhs, h->lam, adj_rtol * bn, &its, &S, &ok,
                 std::max(h->prm.gmres_maxit, kAdjointMaxit));
      if (rc) return rc;
      S.gmres_its += its;
      if (S.newton_its < 32) S.gmres_per_newton[S.newton_its] = its;
      S.newton_its++;  // counts adjoint solves
      if (!ok) return fail(h, TUSAS_ENOCONV, "adjoint GMRES did not converge");
      // grad_eps4 -= lam_n . dF_n/d eps4
      ta = tbeg(h);
      TCK(tusas::elem_run(tusas::M_DEPS, h->ec, Un_, h->Un, nullptr, h->tmp, nullptr, h->st));
      tend(h, TUSAS_T_ADJOINT, ta);
      double d;
      TCK(tusas::multidot(n2, 1, h->lam, 0, h->tmp, h->partials, h->sc + 200, h->st));
      TCK(cudaMemcpyAsync(&d, h->sc + 200, sizeof(double), cudaMemcpyDeviceToHost, h->st));
      TCK(cudaStreamSynchronize(h->st));
      geps -= d;
    }
    // keep U_{n0+1} for the right-hand side of step n0 in the previous segment
    if (k > 0) TCK(cudaMemcpyAsync(h->seg[c + 1], h->seg[1], sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->st));
  }
  // dS/dU_0 = -(dF_1/dU_0)^T lam_1; segment 0 left U_0 in seg[0] and U_1 in seg[1]
  rc = set_state_dev(h, h->seg[0], t0);
  if (rc) return rc;
  TCK(tusas::elem_run(tusas::M_PREV_T, h->ec, h->seg[1], h->Un, h->lam, h->tmp, nullptr, h->st));
  TCK(tusas::vscal(n2, -1.0, h->tmp, h->st));
  if (g0) TCK(tusas::vcopy(n2, h->tmp, g0, h->st));
  if (grad_dir) {
    *grad_dir = 0.0;
    if (d0) {
      TCK(tusas::multidot(n2, 1, h->tmp, 0, d0, h->partials, h->sc + 200, h->st));
      TCK(cudaMemcpyAsync(grad_dir, h->sc + 200, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    }
  }
  // restore the forward's final state
  rc = set_state_dev(h, h->Ufinal, t0 + N * dt);
  if (rc) return rc;
  TCK(cudaStreamSynchronize(h->st));
  *grad_eps4 = geps;
  if (stats) *stats = S;
  return TUSAS_OK;
}

// ---------------------------------------------------------------------------
// Solid fraction S = int (1 + phi_h)/2, the functional of the discrete adjoint
// ---------------------------------------------------------------------------
namespace {
// Integral of the 1D nodal basis function of node i among nnodes: Q1 h (h/2 at
// the two ends); Q2 h/3 at shared element vertices, 2h/3 at midpoints, h/6 at the ends.
__device__ __forceinline__ double sf_weight_1d(int i, int nnodes, int order, double h) {
  if (order == 2) {
    if (i & 1) return 2.0 * h / 3.0;
    return (i == 0 || i == nnodes - 1) ? h / 6.0 : h / 3.0;
  }
  return (i == 0 || i == nnodes - 1) ? 0.5 * h : h;
}

// w = [ (1/2) int psi_node ; 0 ]: S = w^T U + |Omega|/2 (products of 1D integrals on the box)
__global__ void k_sf_weights(tusas::DevMesh m, double* __restrict__ w) {
  for (i64 n = blockIdx.x * (i64)blockDim.x + threadIdx.x; n < m.nn; n += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(n % m.nnx);
    const i64 r = n / m.nnx;
    const int j = (int)(r % m.nny), k = (int)(r / m.nny);
    double v = 0.5 * sf_weight_1d(i, m.nnx, m.order, m.h) * sf_weight_1d(j, m.nny, m.order, m.h);
    if (m.dim == 3) v *= sf_weight_1d(k, m.nnz, m.order, m.h);
    w[n] = v;
    w[m.nn + n] = 0.0;
  }
}
}  // namespace

extern "C" int tusas_solid_fraction(tusas_handle* h, const double* U, double* S, double* w) {
  if (!h) return TUSAS_EINVAL;
  if ((U && !S) || (!U && !w) || (w && w == U)) return fail(h, TUSAS_EINVAL, "bad solid-fraction arguments");
  if (!h->sfw) {
    int rc = ensure_vec(h, &h->sfw);
    if (rc) return rc;
    const i64 nb = std::min<i64>((h->nn + 255) / 256, 148 * 16);
    k_sf_weights<<<(int)nb, 256, 0, h->st>>>(h->dm, h->sfw);
    tusas::count_launches(1);
    TCK(cudaGetLastError());
  }
  if (w) TCK(tusas::vcopy(h->N, h->sfw, w, h->st));
  if (U) {
    TCK(tusas::multidot(h->nn, 1, h->sfw, 0, U, h->partials, h->sc + 200, h->st));
    double v;
    TCK(cudaMemcpyAsync(&v, h->sc + 200, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TCK(cudaStreamSynchronize(h->st));
    const tusas::DevMesh& m = h->dm;
    const double vol = m.h * m.nx * m.h * m.ny * (m.dim == 3 ? m.h * m.nz : 1.0);
    *S = v + 0.5 * vol;
  }
  return TUSAS_OK;
}
