// Element-tile kernels for biquadratic (Q2) elements on 2D structured boxes
// with the 3 x 3 Gauss rule (Sec. 2.1.1; the higher-order discretisation of
// the tip-velocity study, Sec. 4.1): the same operator modes as the Q1 path
// (residual, residual + stored linearisation, tangent, adjoint, dF/d eps4,
// (dF/dU^n)^T w, level-n spatial part) plus the diagonals of the
// preconditioner blocks.
//
// Data path of one CTA (Tile<2> = 16 x 8 elements, one thread per element):
//   1. the tile's 33 x 17 nodes are staged in shared memory (coalesced rows);
//   2. each thread interpolates its element's 9 nodal values to the 9 Gauss
//      points by 1D sum factorisation (3-point Lagrange tables along x, then
//      along y: 135 FMAs for a field's values and gradient instead of 243),
//      evaluates the pointwise integrands of element.cuh, and accumulates the
//      transposed (test-side) sums the same way;
//   3. the element contributions are written to shared memory (reusing the
//      staging buffer) and each tile node sums its <= 4 element contributions
//      in a fixed order before a read-modify-write of the global vector.
// Tiles run in 4 colours (tile-index parity per axis); tiles of one colour
// share no node, so there are no atomics and the result is bitwise
// reproducible.
#include <math.h>

#include "ops.h"

namespace tusas {

struct Q2Args {
  DevMesh m;
  DevPhys P;
  Q2Tab T;
  LinScale Ku;  // unit factors: the Q2 linearisation is stored in true units
  PwConst C;    // pointwise constants, true units
  const double* U;
  const double* Un;
  const double* V;
  double* out;
  double* lin;
  const double* phold;
  int color;
  int ctx, cty;  // tiles of this colour per axis
  int ntx;       // tiles along x (tile id)
};

// Values (and gradients) at the 9 Gauss points g = gx + 3 gy of the field with
// nodal values n[a], a = ax + 3 ay.
template <bool GRAD>
__device__ __forceinline__ void q2_interp(const Q2Tab& T, const double* n, double* val, double* dx, double* dy) {
  double tb[3][3], tg[3][3];  // [gx][ay]
#pragma unroll
  for (int gx = 0; gx < 3; ++gx) {
#pragma unroll
    for (int ay = 0; ay < 3; ++ay) {
      double b = 0.0, d = 0.0;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        b = fma(T.B[gx][ax], n[ax + 3 * ay], b);
        if (GRAD) d = fma(T.G[gx][ax], n[ax + 3 * ay], d);
      }
      tb[gx][ay] = b;
      tg[gx][ay] = d;
    }
  }
#pragma unroll
  for (int gy = 0; gy < 3; ++gy) {
#pragma unroll
    for (int gx = 0; gx < 3; ++gx) {
      double v = 0.0, ddx = 0.0, ddy = 0.0;
#pragma unroll
      for (int ay = 0; ay < 3; ++ay) {
        v = fma(T.B[gy][ay], tb[gx][ay], v);
        if (GRAD) {
          ddx = fma(T.B[gy][ay], tg[gx][ay], ddx);
          ddy = fma(T.G[gy][ay], tb[gx][ay], ddy);
        }
      }
      val[gx + 3 * gy] = v;
      if (GRAD) {
        dx[gx + 3 * gy] = ddx;
        dy[gx + 3 * gy] = ddy;
      }
    }
  }
}

// out_a = sum_g w_g (s_g N_a(g) + fx_g dN_a/dx(g) + fy_g dN_a/dy(g)); with DIAG the
// squared tables give sum_g w_g (s_g N_a^2 + fx_g (dN_a/dx)^2 + fy_g (dN_a/dy)^2).
template <bool DIAG>
__device__ __forceinline__ void q2_accumulate(const Q2Tab& T, const double* s, const double* fx, const double* fy,
                                              double* out) {
  const double(*BW)[3] = DIAG ? T.BB : T.BW;
  const double(*GW)[3] = DIAG ? T.GG : T.GW;
  double t1[3][3], t2[3][3];  // [gx][ay]
#pragma unroll
  for (int gx = 0; gx < 3; ++gx) {
#pragma unroll
    for (int ay = 0; ay < 3; ++ay) {
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int gy = 0; gy < 3; ++gy) {
        a = fma(BW[gy][ay], s[gx + 3 * gy], a);
        a = fma(GW[gy][ay], fy[gx + 3 * gy], a);
        b = fma(BW[gy][ay], fx[gx + 3 * gy], b);
      }
      t1[gx][ay] = a;
      t2[gx][ay] = b;
    }
  }
#pragma unroll
  for (int ay = 0; ay < 3; ++ay) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      double v = 0.0;
#pragma unroll
      for (int gx = 0; gx < 3; ++gx) {
        v = fma(BW[gx][ax], t1[gx][ay], v);
        v = fma(GW[gx][ax], t2[gx][ay], v);
      }
      out[ax + 3 * ay] = v;
    }
  }
}

template <int MODE>
struct Q2MinBlocks {
  static const int V = MODE == M_JV || MODE == M_JTV ? 3 : 2;
};

template <int MODEL, int MODE>
__global__ void __launch_bounds__(Tile<2>::X * Tile<2>::Y, Q2MinBlocks<MODE>::V) q2_kernel(const Q2Args A) {
  constexpr int TX = Tile<2>::X, TY = Tile<2>::Y;
  constexpr int NX = 2 * TX + 1, NY = 2 * TY + 1;
  constexpr int NT = NX * NY;
  constexpr int NE = TX * TY;
  constexpr int NL = 9;  // local nodes = Gauss points
  constexpr int NC = NLin<2, MODEL>::VALUE;
  constexpr bool needU = MODE != M_JV && MODE != M_JTV;
  constexpr bool needV = MODE == M_JV || MODE == M_JTV || MODE == M_PREV_T;
  constexpr int NUF = needU ? 6 : 0;
  constexpr int NVF = needV ? 2 : 0;
  constexpr int NSTAGE = (NUF + NVF) * NT;
  // the next tile colour may start on free SMs now (it waits at the node sums)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  constexpr int NACC = 2 * NL * NE;
  // staging: [NUF][NT] fields phi, u, phi - phi^n, u - u^n, phi^n, phihat_old, then [NVF][NT];
  // after the element arithmetic the same memory holds the contributions [2 NL][NE]
  __shared__ double sm[NSTAGE > NACC ? NSTAGE : NACC];
  double* sU = sm;
  double* sV = sm + NUF * NT;
  double* sC = sm;

  const DevMesh& m = A.m;
  const Q2Tab& T = A.T;
  const int ix = blockIdx.x % A.ctx;
  const int iy = blockIdx.x / A.ctx;
  const int tile_x = 2 * ix + (A.color & 1);
  const int tile_y = 2 * iy + ((A.color >> 1) & 1);
  const int ex0 = tile_x * TX, ey0 = tile_y * TY;
  const int nx0 = 2 * ex0, ny0 = 2 * ey0;
  const bool tf1 = A.P.time_form != 0;

  // ---- 1. stage the tile's nodes --------------------------------------------
  for (int s = threadIdx.x; s < NT; s += NE) {
    const int lx = s % NX, ly = s / NX;
    const int gx = nx0 + lx, gy = ny0 + ly;
    const bool ok = gx < m.nnx && gy < m.nny;
    const i64 node = gx + (i64)m.nnx * gy;
    if (needU) {
      double phi = 0.0, u = 0.0, phin = 0.0, un = 0.0, pho = 0.0;
      if (ok) {
        phi = A.U[node];
        u = A.U[m.nn + node];
        phin = A.Un[node];
        un = A.Un[m.nn + node];
        if (A.phold) pho = A.phold[node];
      }
      sU[0 * NT + s] = phi;
      sU[1 * NT + s] = u;
      sU[2 * NT + s] = phi - phin;
      sU[3 * NT + s] = u - un;
      sU[4 * NT + s] = phin;
      sU[5 * NT + s] = pho;
    }
    if (needV) {
      sV[0 * NT + s] = ok ? A.V[node] : 0.0;
      sV[1 * NT + s] = ok ? A.V[m.nn + node] : 0.0;
    }
  }
  __syncthreads();

  // ---- 2. element arithmetic --------------------------------------------------
  const int t = threadIdx.x;
  const int lx = t % TX, ly = t / TX;
  const int ex = ex0 + lx, ey = ey0 + ly;
  const bool valid = ex < m.nx && ey < m.ny;
  double r0[NL], r1[NL];
#pragma unroll
  for (int a = 0; a < NL; ++a) r0[a] = r1[a] = 0.0;
  if (valid) {
    int sidx[NL];
#pragma unroll
    for (int a = 0; a < NL; ++a) sidx[a] = (2 * lx + a % 3) + NX * (2 * ly + a / 3);
    const i64 tile_id = tile_x + (i64)A.ntx * tile_y;
    double* linp = A.lin + tile_id * (i64)(NC * NL * NE) + t;  // [c][g][t] within the tile
    GPOut<2> o;
    double s0[NL], s1[NL], f0x[NL], f0y[NL], f1x[NL], f1y[NL];
    if (MODE == M_JV || MODE == M_JTV) {
      double n0[NL], n1[NL], v0[NL], v1[NL], v0x[NL], v0y[NL], v1x[NL], v1y[NL];
#pragma unroll
      for (int a = 0; a < NL; ++a) {
        n0[a] = sV[sidx[a]];
        n1[a] = sV[NT + sidx[a]];
      }
      q2_interp<true>(T, n0, v0, v0x, v0y);
      q2_interp<true>(T, n1, v1, v1x, v1y);
#pragma unroll
      for (int g = 0; g < NL; ++g) {
        double L[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) L[c] = __ldg(linp + (c * NL + g) * NE);
        const double xp[2] = {v0x[g], v0y[g]}, xg[2] = {v1x[g], v1y[g]};
        lin_apply<2, MODEL, MODE == M_JTV>(A.P, L, v0[g], v1[g], xp, xg, o);
        s0[g] = o.sphi;
        s1[g] = o.su;
        f0x[g] = o.fphi[0];
        f0y[g] = o.fphi[1];
        f1x[g] = o.fu[0];
        f1y[g] = o.fu[1];
      }
    } else {
      double nd[NL], phi[NL], px[NL], py[NL], u[NL], ux[NL], uy[NL], dphi[NL], du[NL];
#pragma unroll
      for (int a = 0; a < NL; ++a) nd[a] = sU[sidx[a]];
      q2_interp<true>(T, nd, phi, px, py);
#pragma unroll
      for (int a = 0; a < NL; ++a) nd[a] = sU[NT + sidx[a]];
      q2_interp<true>(T, nd, u, ux, uy);
#pragma unroll
      for (int a = 0; a < NL; ++a) nd[a] = sU[2 * NT + sidx[a]];
      q2_interp<false>(T, nd, dphi, nullptr, nullptr);
#pragma unroll
      for (int a = 0; a < NL; ++a) nd[a] = sU[3 * NT + sidx[a]];
      q2_interp<false>(T, nd, du, nullptr, nullptr);
      // grad(phi^n) (literal time term; level-n flux of the theta-method in the adjoint modes)
      const bool oldn = (MODE == M_DEPS || MODE == M_PREV_T) && A.P.theta != 1.0;
      double pnx[NL], pny[NL], pnv[NL];
      if ((tf1 || oldn) && MODE != M_OLD && MODE != M_DIAG) {
#pragma unroll
        for (int a = 0; a < NL; ++a) nd[a] = sU[4 * NT + sidx[a]];
        q2_interp<true>(T, nd, pnv, pnx, pny);
      } else {
#pragma unroll
        for (int g = 0; g < NL; ++g) pnx[g] = pny[g] = 0.0;
      }
      double pho[NL];
      if ((MODE == M_RES || MODE == M_RES_LIN) && A.P.phihat_old) {
#pragma unroll
        for (int a = 0; a < NL; ++a) nd[a] = sU[5 * NT + sidx[a]];
        q2_interp<false>(T, nd, pho, nullptr, nullptr);
      } else {
#pragma unroll
        for (int g = 0; g < NL; ++g) pho[g] = 0.0;
      }
      double w0[NL], w0x[NL], w0y[NL], w1[NL], w1x[NL], w1y[NL], unv[NL], unx[NL], uny[NL];
      if (MODE == M_PREV_T && oldn) {
#pragma unroll
        for (int a = 0; a < NL; ++a) nd[a] = sU[NT + sidx[a]] - sU[3 * NT + sidx[a]];
        q2_interp<true>(T, nd, unv, unx, uny);
      }
      if (MODE == M_PREV_T) {
#pragma unroll
        for (int a = 0; a < NL; ++a) nd[a] = sV[sidx[a]];
        q2_interp<true>(T, nd, w0, w0x, w0y);
#pragma unroll
        for (int a = 0; a < NL; ++a) nd[a] = sV[NT + sidx[a]];
        q2_interp<true>(T, nd, w1, w1x, w1y);
      }
#pragma unroll
      for (int g = 0; g < NL; ++g) {
        const double p[2] = {px[g], py[g]}, gg[2] = {ux[g], uy[g]}, pn[2] = {pnx[g], pny[g]};
        const DevPhys& P = A.P;
        if (MODE == M_DIAG) {
          // Eqs. (pref2), (preconc2) at the Gauss point: mass and stiffness coefficients of M11, M22
          Aniso<2> An;
          An.eval(p, P.eps4);
          const double a2 = An.a * An.a;
          const double B = fma(1.0 - P.k, u[g], 1.0);
          const double phin = phi[g] - dphi[g];
          const double Acoef = MODEL == 0 ? 1.0 : 0.5 * ((1.0 + P.k) - (1.0 - P.k) * phin);
          const double q = MODEL == 0 ? 1.0 : 0.5 * (1.0 - phi[g]);
          s0[g] = P.tau0 * B * a2 * P.idt;
          f0x[g] = f0y[g] = P.thW2 * a2;
          s1[g] = Acoef * P.idt;
          f1x[g] = f1y[g] = P.thD * q;
          continue;
        }
        double G4 = 0.0;
        if (MODEL == 1 && P.has_g4) {
          const double tl = MODE == M_OLD ? P.t_new - P.dt : P.t_new;
          G4 = (fma(m.h, ey + T.xg[g / 3], m.y0) - P.zT - P.Vp * tl) / P.lT;
        }
        if (MODE == M_OLD) {
          spatial_old<2, MODEL>(P, phi[g], u[g], p, gg, G4, o);
        } else if (MODE == M_RES || MODE == M_RES_LIN) {
          double L[MODE == M_RES_LIN ? NC : 1];
          pointwise<2, MODEL, MODE == M_RES_LIN>(P, A.C, phi[g], u[g], dphi[g], du[g], pho[g], p, gg, pn, G4, o, L,
                                                 A.Ku);
          if (MODE == M_RES_LIN) {
#pragma unroll
            for (int c = 0; c < NC; ++c) linp[(c * NL + g) * NE] = L[c];
          }
        } else if (MODE == M_DEPS) {
          gp_deps<2>(P, tf1, phi[g], u[g], dphi[g], du[g], p, pn, o);
        } else {  // M_PREV_T
          const double gw[2] = {w1x[g], w1y[g]};
          gp_prev_t<2, MODEL>(P, tf1, phi[g], u[g], dphi[g], du[g], p, pn, w0[g], w1[g], gw, o);
          if (oldn) {
            const double gn[2] = {unx[g], uny[g]}, gv0[2] = {w0x[g], w0y[g]};
            const double G4n = (MODEL == 1 && P.has_g4)
                                   ? (fma(m.h, ey + T.xg[g / 3], m.y0) - P.zT - P.Vp * (P.t_new - P.dt)) / P.lT
                                   : 0.0;
            old_spatial_t<2, MODEL>(P, phi[g] - dphi[g], u[g] - du[g], pn, gn, G4n, w0[g], gv0, gw, o);
          }
        }
        s0[g] = o.sphi;
        s1[g] = o.su;
        f0x[g] = o.fphi[0];
        f0y[g] = o.fphi[1];
        f1x[g] = o.fu[0];
        f1y[g] = o.fu[1];
      }
    }
    q2_accumulate<MODE == M_DIAG>(T, s0, f0x, f0y, r0);
    q2_accumulate<MODE == M_DIAG>(T, s1, f1x, f1y, r1);
  }
  __syncthreads();  // the contributions overwrite the staging buffer
#pragma unroll
  for (int a = 0; a < NL; ++a) {
    sC[a * NE + t] = r0[a];
    sC[(NL + a) * NE + t] = r1[a];
  }
  __syncthreads();

  // ---- 3. node sums in fixed order, read-modify-write ---------------------------
  // a colour launched as a programmatic dependent of the previous one waits here for that
  // grid's node sums (a no-op after an ordinary launch); the reads bypass L1
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int s = threadIdx.x; s < NT; s += NE) {
    const int nxl = s % NX, nyl = s / NX;
    const int gx = nx0 + nxl, gy = ny0 + nyl;
    if (gx >= m.nnx || gy >= m.nny) continue;
    double acc0 = 0.0, acc1 = 0.0;
    // along each axis a node is local node 2 of element i/2 - 1 and local node 0 of
    // element i/2 (i even), or local node 1 of element (i - 1)/2 (i odd)
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) {
      const int ely = (nyl & 1) ? (cy == 0 ? (nyl - 1) / 2 : -1) : nyl / 2 - 1 + cy;
      const int ay = (nyl & 1) ? 1 : 2 - 2 * cy;
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const int elx = (nxl & 1) ? (cx == 0 ? (nxl - 1) / 2 : -1) : nxl / 2 - 1 + cx;
        const int ax = (nxl & 1) ? 1 : 2 - 2 * cx;
        if (elx >= 0 && elx < TX && ely >= 0 && ely < TY) {
          const int e = elx + TX * ely;
          const int a = ax + 3 * ay;
          acc0 += sC[a * NE + e];
          acc1 += sC[(NL + a) * NE + e];
        }
      }
    }
    const i64 node = gx + (i64)m.nnx * gy;
    A.out[node] = __ldcg(A.out + node) + acc0;
    A.out[m.nn + node] = __ldcg(A.out + m.nn + node) + acc1;
  }
}

void q2_tables(Q2Tab& T, double h) {
  const double s = sqrt(0.6);
  const double xg[3] = {0.5 * (1.0 - s), 0.5, 0.5 * (1.0 + s)};
  const double wg[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  for (int g = 0; g < 3; ++g) {
    const double x = xg[g];
    const double L[3] = {2.0 * (x - 0.5) * (x - 1.0), -4.0 * x * (x - 1.0), 2.0 * x * (x - 0.5)};
    const double dL[3] = {4.0 * x - 3.0, 4.0 - 8.0 * x, 4.0 * x - 1.0};
    T.xg[g] = x;
    for (int a = 0; a < 3; ++a) {
      T.B[g][a] = L[a];
      T.G[g][a] = dL[a] / h;
      T.BW[g][a] = h * wg[g] * L[a];
      T.GW[g][a] = wg[g] * dL[a];
      T.BB[g][a] = h * wg[g] * L[a] * L[a];
      T.GG[g][a] = wg[g] * dL[a] * dL[a] / h;
    }
  }
}

// ---------------------------------------------------------------------------
// Preconditioner blocks M11, M22 (Eqs. pref2, preconc2) of a Q2 box as 25-point
// stencils on its node lattice (spacing h/2): one thread per node gathers the
// rows of the element matrices of its 1, 2 or 4 elements in a fixed order and
// writes its two rows once (no colouring, deterministic). Arithmetic in the
// stencil precision T (the preconditioner's).
// ---------------------------------------------------------------------------
template <typename T>
struct Q2FillArgs {
  DevMesh m;  // the Q2 mesh
  DevPhys P;
  Q2Tab Tb;
  const double* U;
  const double* Un;
  T* st;  // [2][25][nn]
};

template <int MODEL, typename T>
__global__ void __launch_bounds__(256) k_q2_stencil_fill(const Q2FillArgs<T> A) {
  const DevMesh& m = A.m;
  const DevPhys& P = A.P;
  // basis tables in the stencil precision: value, x- and y-derivative of local node b at Gauss point g
  __shared__ T sN[9][9], sNx[9][9], sNy[9][9], sW[9];
  for (int t = threadIdx.x + blockDim.x * threadIdx.y; t < 81; t += blockDim.x * blockDim.y) {
    const int g = t / 9, b = t % 9;
    const int gx = g % 3, gy = g / 3, bx = b % 3, by = b / 3;
    sN[g][b] = T(A.Tb.B[gx][bx] * A.Tb.B[gy][by]);
    sNx[g][b] = T(A.Tb.G[gx][bx] * A.Tb.B[gy][by]);
    sNy[g][b] = T(A.Tb.B[gx][bx] * A.Tb.G[gy][by]);
    if (b == 0) {
      const double wg[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
      sW[g] = T(m.h * m.h * wg[gx] * wg[gy]);
    }
  }
  __syncthreads();
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  const int iy = blockIdx.y * blockDim.y + threadIdx.y;
  if (ix >= m.nnx || iy >= m.nny) return;
  const i64 node = ix + (i64)m.nnx * iy;
  T acc0[25], acc1[25];
#pragma unroll
  for (int o = 0; o < 25; ++o) acc0[o] = acc1[o] = T(0);
  const T k = T(P.k), eps = T(P.eps4), a0 = T(1.0 - 3.0 * P.eps4);
  const T tau_dt = T(P.tau0 * P.idt), idt = T(P.idt), thW2 = T(P.thW2), thD = T(P.thD);
  // candidate elements per axis: even index 2e = right end of e - 1 (local 2) and left end of e
  // (local 0); odd index 2e + 1 = middle of e (local 1)
  for (int cy = 0; cy < 2; ++cy) {
    const int ey = (iy & 1) ? (cy == 0 ? (iy - 1) / 2 : -1) : iy / 2 - 1 + cy;
    const int ay = (iy & 1) ? 1 : 2 - 2 * cy;
    if (ey < 0 || ey >= m.ny) continue;
    for (int cx = 0; cx < 2; ++cx) {
      const int ex = (ix & 1) ? (cx == 0 ? (ix - 1) / 2 : -1) : ix / 2 - 1 + cx;
      const int ax = (ix & 1) ? 1 : 2 - 2 * cx;
      if (ex < 0 || ex >= m.nx) continue;
      const int a = ax + 3 * ay;
      T nphi[9], nu[9], npn[9];
#pragma unroll
      for (int b = 0; b < 9; ++b) {
        const i64 nb = (2 * ex + b % 3) + (i64)m.nnx * (2 * ey + b / 3);
        nphi[b] = narrow<T>(__ldg(A.U + nb));
        nu[b] = narrow<T>(__ldg(A.U + m.nn + nb));
        npn[b] = narrow<T>(__ldg(A.Un + nb));
      }
#pragma unroll 1
      for (int g = 0; g < 9; ++g) {
        T phi = 0, px = 0, py = 0, u = 0, phin = 0;
#pragma unroll
        for (int b = 0; b < 9; ++b) {
          const T Nb = sN[g][b];
          phi += Nb * nphi[b];
          u += Nb * nu[b];
          phin += Nb * npn[b];
          px += sNx[g][b] * nphi[b];
          py += sNy[g][b] * nphi[b];
        }
        // Gauss-point coefficients of the two blocks (as the Q1 fill)
        const T q = px * px + py * py;
        T an = T(1);
        if (q >= T(TUSAS_GUARD_Q)) {
          const T iq = T(1) / q;
          an = a0 + T(4) * eps * (px * px * px * px + py * py * py * py) * iq * iq;
        }
        const T a2 = an * an;
        const T Bu = T(1) + (T(1) - k) * u;
        const T Ac = MODEL == 0 ? T(1) : T(0.5) * ((T(1) + k) - (T(1) - k) * phin);
        const T mob = MODEL == 0 ? T(1) : T(0.5) * (T(1) - phi);
        const T W = sW[g];
        const T Na = sN[g][a], Nax = sNx[g][a], Nay = sNy[g][a];
        const T m0 = W * tau_dt * Bu * a2 * Na, m1 = W * Ac * idt * Na;
        const T k0 = W * thW2 * a2, k1 = W * thD * mob;
        // row of local node a against b = a + (dx, dy): compile-time stencil slots
#pragma unroll
        for (int o = 0; o < 25; ++o) {
          const int bx = ax + o % 5 - 2, by = ay + o / 5 - 2;
          if (bx < 0 || bx > 2 || by < 0 || by > 2) continue;
          const int b = bx + 3 * by;
          const T gd = Nax * sNx[g][b] + Nay * sNy[g][b];
          acc0[o] += m0 * sN[g][b] + k0 * gd;
          acc1[o] += m1 * sN[g][b] + k1 * gd;
        }
      }
    }
  }
#pragma unroll
  for (int o = 0; o < 25; ++o) {
    A.st[(i64)o * m.nn + node] = acc0[o];
    A.st[((i64)25 + o) * m.nn + node] = acc1[o];
  }
}

template <typename T>
cudaError_t q2_stencil_fill(const ElemCtx& c, const double* U, const double* Un, T* st, cudaStream_t s) {
  if (c.m.dim != 2 || c.m.order != 2) return cudaErrorInvalidValue;
  Q2FillArgs<T> a;
  a.m = c.m;
  a.P = c.P;
  a.Tb = c.q2;
  a.U = U;
  a.Un = Un;
  a.st = st;
  const dim3 blk(32, 8);
  const dim3 grid(ceil_div(c.m.nnx, 32), ceil_div(c.m.nny, 8));
  if (c.P.model == 0)
    k_q2_stencil_fill<0, T><<<grid, blk, 0, s>>>(a);
  else
    k_q2_stencil_fill<1, T><<<grid, blk, 0, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}
template cudaError_t q2_stencil_fill<float>(const ElemCtx&, const double*, const double*, float*, cudaStream_t);
template cudaError_t q2_stencil_fill<double>(const ElemCtx&, const double*, const double*, double*, cudaStream_t);

template <int MODEL, int MODE>
static cudaError_t q2_colours(const ElemCtx& c, Q2Args a, cudaStream_t st) {
  constexpr int NE = Tile<2>::X * Tile<2>::Y;
  for (int col = 0; col < 4; ++col) {
    const int cx = col & 1, cy = (col >> 1) & 1;
    a.color = col;
    a.ctx = (c.ntx - cx + 1) / 2;
    a.cty = (c.nty - cy + 1) / 2;
    const long long blocks = (long long)a.ctx * a.cty;
    if (blocks <= 0) continue;
    const cudaError_t e = launch_colour(q2_kernel<MODEL, MODE>, (unsigned)blocks, NE, 0, st, col > 0, a);
    if (e != cudaSuccess) return e;
    count_launches(1);
  }
  return cudaGetLastError();
}

template <int MODEL>
static cudaError_t q2_dispatch(int mode, const ElemCtx& c, const Q2Args& a, cudaStream_t st) {
  switch (mode) {
    case M_RES: return q2_colours<MODEL, M_RES>(c, a, st);
    case M_RES_LIN: return q2_colours<MODEL, M_RES_LIN>(c, a, st);
    case M_JV: return q2_colours<MODEL, M_JV>(c, a, st);
    case M_JTV: return q2_colours<MODEL, M_JTV>(c, a, st);
    case M_DEPS: return q2_colours<MODEL, M_DEPS>(c, a, st);
    case M_PREV_T: return q2_colours<MODEL, M_PREV_T>(c, a, st);
    case M_OLD: return q2_colours<MODEL, M_OLD>(c, a, st);
    case M_DIAG: return q2_colours<MODEL, M_DIAG>(c, a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t q2_run(int mode, const ElemCtx& c, const double* U, const double* Un, const double* V, double* out,
                   double* lin, cudaStream_t st, const double* phold) {
  if (c.m.dim != 2 || c.m.order != 2) return cudaErrorInvalidValue;
  Q2Args a;
  a.m = c.m;
  a.P = c.P;
  a.T = c.q2;
  a.Ku = c.Ku;
  a.C = c.pw_q2;
  a.U = U;
  a.Un = Un;
  a.V = V;
  a.out = out;
  a.lin = lin;
  a.phold = phold;
  a.ntx = c.ntx;
  a.color = 0;
  a.ctx = a.cty = 0;
  return c.P.model == 0 ? q2_dispatch<0>(mode, c, a, st) : q2_dispatch<1>(mode, c, a, st);
}

}  // namespace tusas
