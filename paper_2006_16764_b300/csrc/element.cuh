// Per-element Q1 arithmetic on structured boxes: sum-factorised interpolation
// to the 2^dim Gauss points, the pointwise integrands of the phase-field /
// solute system, their linearisation, and the transposed (test-function)
// accumulation back to the element nodes.
//
// Sum factorisation. The element kernels (FP64) interpolate axis by axis
// (interp_l below): per axis a pair of values gives the two Gauss-point
// values and their difference in three operations, and the test-function
// accumulation is the exact transpose. In 3D this costs 54 FP64 operations
// for the values and gradient of one field at all 8 Gauss points (256 for the
// direct basis sums), which matters because the kernels are bound by the FP64
// pipe, not by memory. The preconditioner fill (FP32 or FP64) interpolates
// with Walsh-Hadamard butterflies (interp): with eta = 2 xi - 1 per axis the
// Q1 interpolant of the element's nodal values v_a (a = ax + 2 ay + 4 az) is
//     v(eta) = 2^-dim sum_b C_b prod_{d in b} eta_d,
// C = H v (butterfly (x, y) -> (x + y, y - x) on every axis); the Gauss points
// sit at eta_d = +-1/sqrt(3), so the values are H^T applied to C_b s^|b| 2^-dim
// (s = 1/sqrt 3), and the derivative along axis d is the (dim-1)-dimensional
// H^T of the coefficients with bit d set, scaled by 2/(h 2^dim) s^(|b|-1).
#pragma once
#include "common.cuh"

namespace tusas {

__host__ __device__ constexpr int insert_bit(int j, int d, int bit) {
  return ((j >> d) << (d + 1)) | (bit << d) | (j & ((1 << d) - 1));
}
__host__ __device__ constexpr int remove_bit(int g, int d) {
  return ((g >> (d + 1)) << d) | (g & ((1 << d) - 1));
}
__host__ __device__ constexpr int popc(int x) { return x == 0 ? 0 : (x & 1) + popc(x >> 1); }

// forward transform H (nodes or Gauss points -> Walsh coefficients)
template <int DIM, typename T = double>
__device__ __forceinline__ void walsh_fwd(T* v) {
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
#pragma unroll
    for (int a = 0; a < (1 << DIM); ++a) {
      if (!(a & (1 << d))) {
        const T x = v[a], y = v[a | (1 << d)];
        v[a] = x + y;
        v[a | (1 << d)] = y - x;
      }
    }
  }
}

// evaluation transform H^T (Walsh coefficients -> values at sign points)
template <int DIM, typename T = double>
__device__ __forceinline__ void walsh_eval(T* v) {
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
#pragma unroll
    for (int a = 0; a < (1 << DIM); ++a) {
      if (!(a & (1 << d))) {
        const T c0 = v[a], c1 = v[a | (1 << d)];
        v[a] = c0 - c1;
        v[a | (1 << d)] = c0 + c1;
      }
    }
  }
}
template <>
__device__ __forceinline__ void walsh_eval<0, double>(double*) {}
template <>
__device__ __forceinline__ void walsh_fwd<0, double>(double*) {}
template <>
__device__ __forceinline__ void walsh_eval<0, float>(float*) {}
template <>
__device__ __forceinline__ void walsh_fwd<0, float>(float*) {}

// Scale factors, computed on the host: value scale vs[k] = s^k 2^-dim,
// gradient scale gs[k] = s^k 2/(h 2^dim); the "w" variants include the Gauss
// weight (h/2)^dim for the accumulation.
template <typename T>
struct ScalesT {
  T vs[4], gs[3], vsw[4], gsw[3];
};
typedef ScalesT<double> Scales;

// Values (and, if GRAD, gradients) of one field at all Gauss points.
// grad[d][j]: derivative along d at the Gauss points whose other-axis bits are j.
template <int DIM, bool GRAD, typename T = double>
__device__ __forceinline__ void interp(const T* nodal, T* val, T (*grad)[1 << (DIM - 1)], const ScalesT<T>& S) {
  constexpr int NN = 1 << DIM;
  T c[NN];
#pragma unroll
  for (int a = 0; a < NN; ++a) c[a] = nodal[a];
  walsh_fwd<DIM, T>(c);
  if (GRAD) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
      for (int j = 0; j < NN / 2; ++j) grad[d][j] = c[insert_bit(j, d, 1)] * S.gs[popc(j)];
      walsh_eval<DIM - 1, T>(grad[d]);
    }
  }
#pragma unroll
  for (int b = 0; b < NN; ++b) val[b] = c[b] * S.vs[popc(b)];
  walsh_eval<DIM, T>(val);
}

// ---- staged 1D forms ----------------------------------------------------------
// Axis by axis, a pair of values (x0 at xi = 0, x1 at xi = 1) gives the values
// at the two Gauss points xi = t and 1 - t, t = (1 - 1/sqrt 3) / 2, and the
// difference b = x1 - x0 (h times the derivative along the axis, constant
// along it): b = x1 - x0, x0 + t b, x1 - t b, three FP64 operations. The
// difference of an earlier axis is carried through the later axes by the same
// two-point interpolation. In 3D this costs 54 operations for the values and
// the 12 distinct gradient entries of a field at the 8 Gauss points (72 with
// the Walsh butterflies of interp), 36 for values alone (56). The
// accumulation is the exact transpose (78 operations against 104): pairs
// (yL, yR) and a derivative term yb go back to the nodes as
// yL - q, yR + q with q = t (yL - yR) + yb.
#define TUSAS_GP_T 0.21132486540518713  // (1 - 1/sqrt(3)) / 2

// Values at the Gauss points and, if GRAD, the differences grad[d][j] = h dv/dx_d at
// the Gauss points whose other-axis bits are j.
template <int DIM, bool GRAD = true>
__device__ __forceinline__ void interp_l(const double* nodal, double* val, double (*grad)[1 << (DIM - 1)]) {
  constexpr int NN = 1 << DIM;
  constexpr int NH = NN / 2;
  const double t = TUSAS_GP_T;
#pragma unroll
  for (int a = 0; a < NN; ++a) val[a] = nodal[a];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    if (GRAD) {
#pragma unroll
      for (int e = 0; e < d; ++e) {  // earlier differences: axis d is bit d - 1 of j
#pragma unroll
        for (int j = 0; j < NH; ++j) {
          if (!(j & (1 << (d - 1)))) {
            const double x0 = grad[e][j], x1 = grad[e][j | (1 << (d - 1))];
            const double b = x1 - x0;
            grad[e][j] = fma(t, b, x0);
            grad[e][j | (1 << (d - 1))] = fma(-t, b, x1);
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      if (!(a & (1 << d))) {
        const double x0 = val[a], x1 = val[a | (1 << d)];
        const double b = x1 - x0;
        if (GRAD) grad[d][remove_bit(a, d)] = b;
        val[a] = fma(t, b, x0);
        val[a | (1 << d)] = fma(-t, b, x1);
      }
    }
  }
}

// Values and gradients in true units (the differences of interp_l times 1/h).
template <int DIM, bool GRAD>
__device__ __forceinline__ void interp_true(const double* nodal, double* val, double (*grad)[1 << (DIM - 1)],
                                            double inv_h) {
  interp_l<DIM, GRAD>(nodal, val, grad);
  if (GRAD) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
      for (int j = 0; j < (1 << (DIM - 1)); ++j) grad[d][j] *= inv_h;
    }
  }
}

// Transpose of interp_l: out_a = sum_g ( sv_g N_a(g) + sum_d f_dg h dN_a/dx_d(g) ).
// The fluxes f[d][g] are summed over the two Gauss points along d first (the
// difference along d is the same at both).
template <int DIM>
__device__ __forceinline__ void accumulate_l(const double* sv, double (*f)[1 << DIM], double* out) {
  constexpr int NN = 1 << DIM;
  constexpr int NH = NN / 2;
  const double t = TUSAS_GP_T;
  double F[DIM][NH];
#pragma unroll
  for (int a = 0; a < NN; ++a) out[a] = sv[a];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
#pragma unroll
    for (int j = 0; j < NH; ++j) F[d][j] = f[d][insert_bit(j, d, 0)] + f[d][insert_bit(j, d, 1)];
  }
#pragma unroll
  for (int d = DIM - 1; d >= 0; --d) {
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      if (!(a & (1 << d))) {
        const double yL = out[a], yR = out[a | (1 << d)];
        const double q = fma(t, yL - yR, F[d][remove_bit(a, d)]);
        out[a] = yL - q;
        out[a | (1 << d)] = yR + q;
      }
    }
#pragma unroll
    for (int e = 0; e < d; ++e) {
#pragma unroll
      for (int j = 0; j < NH; ++j) {
        if (!(j & (1 << (d - 1)))) {
          const double yL = F[e][j], yR = F[e][j | (1 << (d - 1))];
          const double dd = yL - yR;
          F[e][j] = fma(-t, dd, yL);
          F[e][j | (1 << (d - 1))] = fma(t, dd, yR);
        }
      }
    }
  }
}

// Factors of the stored linearisation for the staged forms, by the type of a
// coefficient: (input value | gradient) -> (output value | flux). interp_l gives
// values and h times the gradients; accumulate_l takes values times the Gauss
// weight w and fluxes times w / h, so vv = w, gv = vf = w / h, gf = w / h^2.
// The same stored coefficients then serve the transposed product unchanged.
// Also the model-0 constants of the u equation, scaled.
#define TUSAS_INV_2SQRT2 0.35355339059327373

struct LinScale {
  double vv, gv, vf, gf;
  double mdphat, idt, thD;
  // physics constants times their factors, for the linearisation pass (lin_consts)
  double m_th_vv, tau_idt_vv, thlam_vv, tau_vv, tau2_gv, thW2_gf, half_omk_vv, m_half_thD_vf, cw_dphat_vf, cw_omk_vf,
      half_thD_gf, cw_gf;
};

// Fill the linearisation constants of K from the physics P (host).
inline void lin_consts(LinScale& K, const DevPhys& P) {
  const double cw = TUSAS_INV_2SQRT2 * P.W0, omk = 1.0 - P.k;
  K.mdphat = -0.5 * P.dphat * K.vv;
  K.idt = P.idt * K.vv;
  K.thD = P.thD * K.gf;
  K.m_th_vv = -P.theta * K.vv;
  K.tau_idt_vv = P.tau0 * P.idt * K.vv;
  K.thlam_vv = P.theta * P.lam * K.vv;
  K.tau_vv = P.tau0 * K.vv;
  K.tau2_gv = 2.0 * P.tau0 * K.gv;
  K.thW2_gf = P.thW2 * K.gf;
  K.half_omk_vv = 0.5 * omk * K.vv;
  K.m_half_thD_vf = -0.5 * P.thD * K.vf;
  K.cw_dphat_vf = cw * P.dphat * K.vf;
  K.cw_omk_vf = cw * omk * K.vf;
  K.half_thD_gf = 0.5 * P.thD * K.gf;
  K.cw_gf = cw * K.gf;
}

// ---------------------------------------------------------------------------
// Pointwise physics (Sec. 4.2, Eqs. pf2, lambda, directional, conc2, jat, gs)
// ---------------------------------------------------------------------------

#define TUSAS_GUARD_Q 1e-20

// Anisotropy a(p) = 1 - 3 eps + 4 eps sum n_i^4 (Eq. gs) from p = grad phi.
// On return n[] is the unit normal, n2[] its squares, sn = sum n_i^4, r = 1/|p|
// (all zero and a = 1 where |p|^2 < 1e-20).
template <int DIM>
struct Aniso {
  double a, sn, r;
  double n[DIM], n2[DIM];
  // guard_q: the guard threshold on |p|^2 in the units of p (1e-20 for true gradients)
  __device__ __forceinline__ void eval(const double* p, double eps, double guard_q = TUSAS_GUARD_Q) {
    double q = p[0] * p[0];
#pragma unroll
    for (int d = 1; d < DIM; ++d) q = fma(p[d], p[d], q);
    if (q < guard_q) {
      a = 1.0;
      sn = 0.0;
      r = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) n[d] = n2[d] = 0.0;
    } else {
      r = rsqrt(q);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        n[d] = p[d] * r;
        n2[d] = n[d] * n[d];
      }
      sn = n2[0] * n2[0];
#pragma unroll
      for (int d = 1; d < DIM; ++d) sn = fma(n2[d], n2[d], sn);
      a = fma(4.0 * eps, sn, 1.0 - 3.0 * eps);
    }
  }
};

// Integrands at one Gauss point.
template <int DIM>
struct GPOut {
  double sphi, fphi[DIM], su, fu[DIM];
};

// Number of stored linearisation coefficients per Gauss point.
template <int DIM, int MODEL>
struct NLin {
  static const int SYM = DIM * (DIM + 1) / 2;
  static const int PHI = 2 + DIM + SYM;              // alpha_phi, alpha_u, alpha_p, H
  // alloy: beta_phi, beta_u, gamma_phi, c_u, gamma_g, kappa1, nvec (the second antitrapping
  // factor kappa2 is kappa1 for the normalised current and 0 for the printed one: not stored)
  static const int VALUE = MODEL == 0 ? PHI : PHI + 2 + DIM + 3 + DIM;
};

// unit factors: stored coefficients in true units (host)
inline LinScale lin_unit(const DevPhys& P) {
  LinScale K{};
  K.vv = K.gv = K.vf = K.gf = 1.0;
  lin_consts(K, P);
  return K;
}

// Constants of pointwise() for gradients given as gsc times the true gradient (true
// units: gsc = 1; the staged forms of the 3D tile residual pass h-scaled differences,
// gsc = 1/h), with the linearisation factors K. Where a gradient enters linearly its unit
// rides on a uniform constant, and 1/|p| is rescaled the same way, so the integrands cost
// no conversions per Gauss point. Also the frozen gradient G4 = z ilT + g4off.
struct PwConst {
  double guard_q;   // small-gradient guard on |p|^2 in the caller's units: 1e-20 / gsc^2
  double gsc;       // true gradient = gsc x caller gradient
  double thW2g;     // theta W0^2 gsc
  double thDg;      // theta D gsc (pure-metal diffusion flux)
  double halfthDg;  // theta D gsc / 2 (alloy: D q(phi) grad u)
  double cw, cwg;   // W0/(2 sqrt 2): antitrapping along n; and times gsc, along the printed grad phi
  double tau2c;     // K.tau2_gv 16 eps / gsc: alpha_p = tau2c B (phi - phi^n)/dt a / |p_caller| R
  double kapc;      // K.cw_gf / gsc: kappa = kapc B phihat / |p_caller|
  double mhthDg;    // K.m_half_thD_vf gsc: gamma_phi = mhthDg grad u_caller + ...
  double e32g, e256g;  // K.thW2_gf 32 eps, K.thW2_gf 256 eps^2 (flux Hessian)
  double thW2gf;    // K.thW2_gf
  double ilT, g4off;   // G4 = z / lT - (zT + Vp t^{n+1}) / lT
  double tauidt;    // tau0 / dt
  double a_idt, ma_idt;  // A(phi^n) / dt = a_idt + ma_idt phi^n: (1 + k) / (2 dt), -(1 - k) / (2 dt)
};

inline PwConst pw_consts(const DevPhys& P, const LinScale& K, double gsc) {
  PwConst c{};
  c.guard_q = TUSAS_GUARD_Q / (gsc * gsc);
  c.gsc = gsc;
  c.thW2g = P.thW2 * gsc;
  c.thDg = P.thD * gsc;
  c.halfthDg = 0.5 * P.thD * gsc;
  c.cw = TUSAS_INV_2SQRT2 * P.W0;
  c.cwg = c.cw * gsc;
  c.tau2c = K.tau2_gv * 16.0 * P.eps4 / gsc;
  c.kapc = K.cw_gf / gsc;
  c.mhthDg = K.m_half_thD_vf * gsc;
  c.e32g = K.thW2_gf * 32.0 * P.eps4;
  c.e256g = K.thW2_gf * 256.0 * P.eps4 * P.eps4;
  c.thW2gf = K.thW2_gf;
  c.ilT = P.has_g4 ? 1.0 / P.lT : 0.0;
  c.g4off = P.has_g4 ? -(P.zT + P.Vp * P.t_new) / P.lT : 0.0;
  c.tauidt = P.tau0 * P.idt;
  c.a_idt = 0.5 * (1.0 + P.k) * P.idt;
  c.ma_idt = -0.5 * (1.0 - P.k) * P.idt;
  return c;
}

// symmetric index (i <= j) -> 0..SYM-1: diagonal first, then (0,1),(0,2),(1,2)
template <int DIM>
__host__ __device__ constexpr int sym_index(int i, int j) {
  return i == j ? i : (DIM == 2 ? 2 : (i + j == 1 ? 3 : (i + j == 2 ? 4 : 5)));
}

// Residual integrands and, if LIN, the pointwise Jacobian written to L[c]
// (c-th coefficient of this Gauss point; stride given by the caller's writer).
// p, g, pn are the gradients of phi, u, phi^n in the caller's units (C.gsc times
// them is the true gradient); the outputs are in true units: sphi, su the
// source terms, fphi, fu the fluxes. The stored coefficients L carry the
// LinScale factors of their type (K; unit factors give the coefficients in true
// units): the factors ride on constants that are uniform across threads, so
// they cost no work per Gauss point. The pure metal (MODEL 0) has k = 1, so
// B(u) = 1 and A(phi^n) = 1 are constants there.
template <int DIM, int MODEL, bool LIN>
__device__ __forceinline__ void pointwise(const DevPhys& P, const PwConst& C, double phi, double u, double dphi,
                                          double du, double phold, const double* p, const double* g,
                                          const double* pn, double G4, GPOut<DIM>& o, double* L,
                                          const LinScale& K) {
  Aniso<DIM> A;
  A.eval(p, P.eps4, C.guard_q);
  const double eps = P.eps4;
  const double c16 = 16.0 * eps;
  // anisotropic flux f = theta W0^2 a p_i (a + 16 eps (n_i^2 - sn)), the last factor as
  // 16 eps n_i^2 + (a - 16 eps sn)
  const double W2a = C.thW2g * A.a;
  const double aa = fma(-c16, A.sn, A.a);
#pragma unroll
  for (int d = 0; d < DIM; ++d) o.fphi[d] = W2a * p[d] * fma(c16, A.n2[d], aa);
  const double omk = 1.0 - P.k;
  const double B = MODEL == 0 ? 1.0 : fma(omk, u, 1.0);
  const double Bd = MODEL == 0 ? dphi : B * dphi;  // B (phi - phi^n)
  const double Bt = Bd * P.idt;                     // B (phi - phi^n) / dt
  // phihat of the u source and of j: (phi - phi^n)/dt, or the Eq. (theta) estimate; Bp = B phihat
  double Bp = Bt, phihat = 0.0;
  if (P.phihat_old) {
    phihat = fma(P.theta, dphi * P.idt, (1.0 - P.theta) * phold);
    Bp = MODEL == 0 ? phihat : B * phihat;
  } else if (LIN) {
    phihat = dphi * P.idt;
  }
  const double a2 = A.a * A.a;
  const double om = fma(-phi, phi, 1.0);  // 1 - phi^2
  const double ug = u + G4;
  const double phom = phi * om;
  const double om2 = om * om;
  const double phin = phi - dphi;
  double time;
  if (P.time_form == 0) {
    time = (a2 * C.tauidt) * Bd;  // tau0 a^2 B (phi - phi^n) / dt
  } else {
    Aniso<DIM> An;
    An.eval(pn, eps, C.guard_q);
    const double Bn = MODEL == 0 ? 1.0 : fma(omk, u - du, 1.0);
    time = P.tau0 * (B * a2 * phi - Bn * (An.a * An.a) * phin) * P.idt;
  }
  o.sphi = fma(-P.theta, fma(-P.lam * om2, ug, phom), time);
  const double Ai = MODEL == 0 ? P.idt : fma(C.ma_idt, phin, C.a_idt);  // A(phi^n) / dt
  o.su = fma(-0.5, Bp, Ai * du);
  double Bpr = 0.0;
  if (MODEL == 0) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) o.fu[d] = C.thDg * g[d];
  } else {
    const double Dq = fma(-C.halfthDg, phi, C.halfthDg);  // theta D (1 - phi) / 2
    Bpr = Bp * A.r;
    const double jn = P.jat_norm ? C.cw * Bpr : C.cwg * Bp;
#pragma unroll
    for (int d = 0; d < DIM; ++d) o.fu[d] = fma(Dq, g[d], jn * p[d]);
  }
  if constexpr (LIN) {
    // ---- pointwise Jacobian -------------------------------------------------
    // m_i = n_i^2 - sn, R_i = n_i m_i: da/dp_i = 16 eps R_i / |p|
    double m[DIM], R[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      m[d] = A.n2[d] - A.sn;
      R[d] = A.n[d] * m[d];
    }
    const double phi2 = phi * phi;
    const double dbulk = fma(4.0 * P.lam * phom, ug, fma(-3.0, phi2, 1.0));
    // with the literal time term the coefficients of d(B a^2) multiply phi/dt instead of phihat
    const double tfac = P.time_form == 0 ? dphi * P.idt : phi * P.idt;
    const double Btf = P.time_form == 0 ? Bt : (MODEL == 0 ? tfac : B * tfac);
    L[0] = fma(K.m_th_vv, dbulk, K.tau_idt_vv * B * a2);  // alpha_phi
    L[1] = MODEL == 0 ? K.thlam_vv * om2 : fma(K.thlam_vv, om2, K.tau_vv * omk * a2 * tfac);  // alpha_u
    const double c2a = C.tau2c * Btf * (A.a * A.r);
#pragma unroll
    for (int d = 0; d < DIM; ++d) L[2 + d] = c2a * R[d];  // alpha_p = 2 tau0 B a da/dp
    // H = theta W0^2 [ delta_ij (a^2 + 16 eps a (3 n_i^2 - sn)) + n_i n_j B_ij ],
    //   B_ij = 256 eps^2 m_i m_j - 32 eps a (m_i + m_j + sn); n_i n_j B_ij = P_i R_j - T_i n_j with
    //   P_i = n_i (256 eps^2 m_i - 32 eps a), T_i = 32 eps a n_i^3; the diagonal term is
    //   a^2 + 32 eps a sn + 48 eps a m_i. theta W0^2 and the coefficient factor ride on the constants.
    const double kt = C.e32g * A.a;
    const double kd0 = fma(kt, A.sn, C.thW2gf * a2), kd1 = 1.5 * kt;
    double Pk[DIM], Tk[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      Pk[i] = A.n[i] * fma(C.e256g, m[i], -kt);
      Tk[i] = kt * (A.n[i] * A.n2[i]);
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
#pragma unroll
      for (int j = i; j < DIM; ++j) {
        double v = fma(Pk[i], R[j], -Tk[i] * A.n[j]);
        if (i == j) v += fma(kd1, m[i], kd0);
        L[2 + DIM + sym_index<DIM>(i, j)] = v;
      }
    }
    if (MODEL == 1) {
      constexpr int o0 = NLin<DIM, 1>::PHI;
      L[o0 + 0] = K.mdphat * B;                            // beta_phi
      L[o0 + 1] = fma(Ai, K.vv, -K.half_omk_vv * phihat);  // beta_u = (A(phi^n)/dt - (1-k) phihat / 2) vv
      // direction of the antitrapping current (true units) and its derivative factors
      double nv[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) nv[d] = P.jat_norm ? A.n[d] : C.gsc * p[d];
      const double kap = P.jat_norm ? C.kapc * Bpr : K.cw_gf * Bp;
      const double cgp = K.cw_dphat_vf * B;
#pragma unroll
      for (int d = 0; d < DIM; ++d) L[o0 + 2 + d] = fma(C.mhthDg, g[d], cgp * nv[d]);  // gamma_phi
      L[o0 + 2 + DIM] = K.cw_omk_vf * phihat;                                           // c_u
      L[o0 + 3 + DIM] = fma(-K.half_thD_gf, phi, K.half_thD_gf);                        // gamma_g
      L[o0 + 4 + DIM] = kap;                                                            // kappa1
#pragma unroll
      for (int d = 0; d < DIM; ++d) L[o0 + 5 + DIM + d] = nv[d];  // nvec
    }
  }
}

// Level-n spatial integrands weighted (1 - theta) (theta-method, Eqs. dpf / dc):
// -(1-theta) bulk(phi^n, u^n, G4(t^n)), (1-theta) f_phi(grad phi^n), (1-theta) D q(phi^n) grad u^n.
template <int DIM, int MODEL>
__device__ __forceinline__ void spatial_old(const DevPhys& P, double phi, double u, const double* p, const double* g,
                                            double G4, GPOut<DIM>& o) {
  const double w = 1.0 - P.theta;
  Aniso<DIM> A;
  A.eval(p, P.eps4);
  const double c16 = 16.0 * P.eps4;
  const double W2a = w * P.W0 * P.W0 * A.a;
#pragma unroll
  for (int d = 0; d < DIM; ++d) o.fphi[d] = W2a * p[d] * fma(c16, A.n2[d] - A.sn, A.a);
  const double om = 1.0 - phi * phi;
  o.sphi = -w * (phi * om - P.lam * om * om * (u + G4));
  o.su = 0.0;
  const double Dq = MODEL == 0 ? w * P.D : 0.5 * w * P.D * (1.0 - phi);
#pragma unroll
  for (int d = 0; d < DIM; ++d) o.fu[d] = Dq * g[d];
}

// d/d eps4 of the anisotropic flux W^2 a(p) (a + 16 eps (n_i^2 - sn)) p_i, scaled by w.
template <int DIM>
__device__ __forceinline__ void flux_deps(const DevPhys& P, const double* p, double w, double* f) {
  Aniso<DIM> An;
  An.eval(p, P.eps4);
  const double ae = An.r == 0.0 ? 0.0 : fma(4.0, An.sn, -3.0);
  const double W2 = w * P.W0 * P.W0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const double md = An.n2[d] - An.sn;
    f[d] += W2 * p[d] * (ae * fma(16.0 * P.eps4, md, An.a) + An.a * fma(16.0, md, ae));
  }
}

// d(integrands)/d eps4 at one Gauss point (Eq. gs differentiated in eps4, through
// the flux and the tau(n) time term). tf1: difference-of-products time term; pn is
// grad(phi^n), used by tf1 and, for theta < 1, by the level-n flux weighted (1 - theta).
template <int DIM>
__device__ __forceinline__ void gp_deps(const DevPhys& P, bool tf1, double phi, double u, double dphi, double du,
                                        const double* p, const double* pn, GPOut<DIM>& o) {
  Aniso<DIM> An;
  An.eval(p, P.eps4);
  const double ae = An.r == 0.0 ? 0.0 : fma(4.0, An.sn, -3.0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) o.fphi[d] = o.fu[d] = 0.0;
  flux_deps<DIM>(P, p, P.theta, o.fphi);
  if (P.theta != 1.0) flux_deps<DIM>(P, pn, 1.0 - P.theta, o.fphi);
  const double B = fma(1.0 - P.k, u, 1.0);
  if (!tf1) {
    o.sphi = P.tau0 * B * dphi * P.idt * 2.0 * An.a * ae;
  } else {
    Aniso<DIM> Ao;
    Ao.eval(pn, P.eps4);
    const double aoe = Ao.r == 0.0 ? 0.0 : fma(4.0, Ao.sn, -3.0);
    const double Bn = fma(1.0 - P.k, u - du, 1.0);
    o.sphi = P.tau0 * P.idt * 2.0 * (B * An.a * ae * phi - Bn * Ao.a * aoe * (phi - dphi));
  }
  o.su = 0.0;
}

// Transposed linearisation of the level-n spatial integrands weighted (1 - theta)
// (spatial_old) at (phi^n, u^n, grad phi^n = pn, grad u^n = gn, G4 at t^n), applied to
// the adjoint fields (w0, grad w0 = gw0, w1, grad w1 = gw1) and added to o.
template <int DIM, int MODEL>
__device__ __forceinline__ void old_spatial_t(const DevPhys& P, double phin, double un, const double* pn,
                                              const double* gn, double G4, double w0, const double* gw0,
                                              const double* gw1, GPOut<DIM>& o) {
  const double wt = 1.0 - P.theta;
  Aniso<DIM> A;
  A.eval(pn, P.eps4);
  const double eps = P.eps4, a2 = A.a * A.a;
  const double om = 1.0 - phin * phin;
  // -d(bulk)/d phi and -d(bulk)/d u, bulk = phi - phi^3 - lam (1 - phi^2)^2 (u + G4)
  const double sphi = -((1.0 - 3.0 * phin * phin) + 4.0 * P.lam * phin * om * (un + G4));
  const double su = P.lam * om * om;
  const double qp = MODEL == 0 ? 0.0 : -0.5 * P.D;  // D dq/dphi
  const double q = MODEL == 0 ? P.D : 0.5 * P.D * (1.0 - phin);
  double gdot = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) gdot = fma(gn[d], gw1[d], gdot);
  o.sphi = fma(wt, fma(sphi, w0, qp * gdot), o.sphi);
  o.su = fma(wt * su, w0, o.su);
  // flux Hessian, as in pointwise()
  const double e32a = 32.0 * eps * A.a, e256 = 256.0 * eps * eps, e16a = 16.0 * eps * A.a;
  const double W2 = wt * P.W0 * P.W0;
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    double hx = 0.0;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const double mi = A.n2[i] - A.sn, mj = A.n2[j] - A.sn;
      double v = A.n[i] * A.n[j] * (e32a * (A.sn - A.n2[i] - A.n2[j]) + e256 * mi * mj);
      if (i == j) v += a2 + e16a * (3.0 * A.n2[i] - A.sn);
      hx = fma(v, gw0[j], hx);
    }
    o.fphi[i] = fma(W2, hx, o.fphi[i]);
    o.fu[i] = fma(wt * q, gw1[i], o.fu[i]);
  }
}

// Integrands of (dF/dU^n)^T w at one Gauss point: (w0, w1) the values of the
// two adjoint fields there, gw1 the gradient of w1.
template <int DIM, int MODEL>
__device__ __forceinline__ void gp_prev_t(const DevPhys& P, bool tf1, double phi, double u, double dphi, double du,
                                          const double* p, const double* pn, double w0, double w1,
                                          const double* gw1, GPOut<DIM>& o) {
  Aniso<DIM> An;
  An.eval(p, P.eps4);
  const double omk = 1.0 - P.k;
  const double B = fma(omk, u, 1.0);
  const double phin = phi - dphi;
  double ds_dpn, ds_dun = 0.0, cpn = 0.0, apn[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) apn[d] = 0.0;
  if (!tf1) {
    ds_dpn = -P.tau0 * B * An.a * An.a * P.idt;
  } else {
    Aniso<DIM> Ao;
    Ao.eval(pn, P.eps4);
    const double Bn = fma(omk, u - du, 1.0);
    ds_dpn = -P.tau0 * Bn * Ao.a * Ao.a * P.idt;
    ds_dun = -P.tau0 * omk * Ao.a * Ao.a * phin * P.idt;
    cpn = -2.0 * P.tau0 * Bn * phin * P.idt * Ao.a;
#pragma unroll
    for (int d = 0; d < DIM; ++d) apn[d] = 16.0 * P.eps4 * Ao.n[d] * (Ao.n2[d] - Ao.sn) * Ao.r;
  }
  const double Acoef = MODEL == 0 ? 1.0 : 0.5 * ((1.0 + P.k) - omk * phin);
  const double dsu_dpn = -0.5 * omk * du * P.idt + 0.5 * B * P.idt;
  const double dsu_dun = -Acoef * P.idt;
  double jp = 0.0;
  if (MODEL == 1) {
    const double cw = -TUSAS_INV_2SQRT2 * P.W0 * B * P.idt;
    double nfu = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) nfu = fma(P.jat_norm ? An.n[d] : p[d], gw1[d], nfu);
    jp = cw * nfu;
  }
  o.sphi = ds_dpn * w0 + dsu_dpn * w1 + jp;
  o.su = ds_dun * w0 + dsu_dun * w1;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    o.fphi[d] = cpn * apn[d] * w0;
    o.fu[d] = 0.0;
  }
}

// Apply the stored pointwise Jacobian (TRANS = false) or its transpose.
// Inputs (x0, x1, xp, xg): forward = (dphi, du, dp, dg);
// transpose = (s_phi, s_u, f_phi, f_u) test-side quantities.
// SCALED: L, the inputs and the outputs are in the staged forms (interp_l /
// accumulate_l, LinScale K); otherwise in true units (K unused).
template <int DIM, int MODEL, bool TRANS, bool SCALED = false>
__device__ __forceinline__ void lin_apply(const DevPhys& P, const double* L, double x0, double x1, const double* xp,
                                          const double* xg, GPOut<DIM>& o, const LinScale& K = LinScale{}) {
  const double mdphat = SCALED ? K.mdphat : -0.5 * P.dphat;
  const double idt = SCALED ? K.idt : P.idt;
  const double thD = SCALED ? K.thD : P.thD;
  constexpr int S0 = 2 + DIM;
  double Hx[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < DIM; ++j) v = fma(L[S0 + sym_index<DIM>(i < j ? i : j, i < j ? j : i)], xp[j], v);
    Hx[i] = v;
  }
  if (!TRANS) {
    double sp = fma(L[0], x0, L[1] * x1);
#pragma unroll
    for (int d = 0; d < DIM; ++d) sp = fma(L[2 + d], xp[d], sp);
    o.sphi = sp;
#pragma unroll
    for (int d = 0; d < DIM; ++d) o.fphi[d] = Hx[d];
    if (MODEL == 0) {
      o.su = fma(mdphat, x0, x1 * idt);
#pragma unroll
      for (int d = 0; d < DIM; ++d) o.fu[d] = thD * xg[d];
    } else {
      constexpr int o0 = NLin<DIM, 1>::PHI;
      o.su = fma(L[o0], x0, L[o0 + 1] * x1);
      const double* nv = L + o0 + 5 + DIM;
      double ndp = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) ndp = fma(nv[d], xp[d], ndp);
      const double k2 = P.jat_norm ? L[o0 + 4 + DIM] : 0.0;  // kappa2
      const double cu = L[o0 + 2 + DIM] * x1 - k2 * ndp;
#pragma unroll
      for (int d = 0; d < DIM; ++d)
        o.fu[d] = fma(L[o0 + 2 + d], x0, fma(L[o0 + 3 + DIM], xg[d], fma(L[o0 + 4 + DIM], xp[d], cu * nv[d])));
    }
  } else {
    // x0 = s_phi-hat, x1 = s_u-hat, xp = f_phi-hat, xg = f_u-hat
    double s0 = L[0] * x0, s1 = L[1] * x0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) o.fphi[d] = fma(L[2 + d], x0, Hx[d]);
    if (MODEL == 0) {
      s0 = fma(mdphat, x1, s0);
      s1 = fma(idt, x1, s1);
#pragma unroll
      for (int d = 0; d < DIM; ++d) o.fu[d] = thD * xg[d];
    } else {
      constexpr int o0 = NLin<DIM, 1>::PHI;
      const double* nv = L + o0 + 5 + DIM;
      s0 = fma(L[o0], x1, s0);
      s1 = fma(L[o0 + 1], x1, s1);
      double nfu = 0.0, gs = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        gs = fma(L[o0 + 2 + d], xg[d], gs);
        nfu = fma(nv[d], xg[d], nfu);
      }
      s0 += gs;
      s1 = fma(L[o0 + 2 + DIM], nfu, s1);
      const double k2 = (P.jat_norm ? L[o0 + 4 + DIM] : 0.0) * nfu;  // kappa2 (n . f_u)
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        o.fphi[d] = fma(L[o0 + 4 + DIM], xg[d], fma(-k2, nv[d], o.fphi[d]));
        o.fu[d] = L[o0 + 3 + DIM] * xg[d];
      }
    }
    o.sphi = s0;
    o.su = s1;
  }
}

}  // namespace tusas
