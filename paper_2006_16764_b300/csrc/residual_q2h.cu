// Element-tile kernels for triquadratic (Q2) hexahedra on 3D structured boxes
// with the 3 x 3 x 3 Gauss rule (Sec. 2.1.1, the higher-order elements of the
// tip-velocity study, Sec. 4.1, in three dimensions): the operator modes of
// the Q1 path (residual, residual + stored linearisation, tangent, adjoint,
// dF/d eps4, (dF/dU^n)^T w, level-n spatial part) and the diagonals of the
// preconditioner blocks.
//
// Data path of one CTA (Q2HexTile = 4 x 2 x 2 elements, one warp per element):
//   1. the tile's 9 x 5 x 5 nodes are staged in shared memory;
//   2. the warp interpolates its element's fields to the 27 Gauss points by
//      sum factorisation spread over the lanes: lane l = i0 + 3 i1 + 9 i2
//      first contracts a node line along x (Gauss point i0, node row
//      (i1, i2)), then the lanes exchange these partial sums by shuffles
//      for the contraction along y and along z, so that lane l ends with
//      the value and gradient at Gauss point (i0, i1, i2): 27 FP64 FMAs per
//      lane and field (729 per element, the cost of full sum factorisation,
//      against 2916 for direct basis sums);
//   3. each lane evaluates the pointwise integrands of its Gauss point
//      (element.cuh) and the transposed stages (z, y, x) bring the test-side
//      sums back to the lanes, lane l now holding the contribution to local
//      node (i0, i1, i2);
//   4. contributions go to shared memory and each tile node sums its <= 8
//      element contributions in a fixed order before a read-modify-write of
//      the global vector. Tiles run in 8 colours (tile-index parity per
//      axis), so no atomics and bitwise reproducible results.
// Lanes 27..31 mirror lane 26 and are never read.
#include <math.h>

#include "ops.h"

namespace tusas {

namespace {
constexpr int HX = Q2HexTile::X, HY = Q2HexTile::Y, HZ = Q2HexTile::Z;
constexpr int HNE = HX * HY * HZ;  // elements (warps) per tile
constexpr int HNX = 2 * HX + 1, HNY = 2 * HY + 1, HNZ = 2 * HZ + 1;
constexpr int HNT = HNX * HNY * HNZ;  // staged nodes per field
constexpr int HTHREADS = 32 * HNE;
constexpr unsigned FULL = 0xffffffffu;
}  // namespace

struct Q2HArgs {
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
  int ctx, cty, ctz;  // tiles of this colour per axis
  int ntx, nty;       // tiles per axis (tile id)
};

// 1D tables in shared memory (lane-dependent indices)
struct Q2HTab {
  double B[3][3], G[3][3], BW[3][3], GW[3][3], BB[3][3], GG[3][3];
};

// Value (and gradient) at Gauss point (i0, i1, i2) of the field staged at sN, element
// corner node `nb` of the tile (see the file comment). Warp-uniform call.
// SY, SZ: strides of the staged node array along y and z (the tile's, by default).
template <bool GRAD, int SY = HNX, int SZ = HNX * HNY>
__device__ __forceinline__ void q2h_interp(const Q2HTab& T, const double* sN, int nb, int i0, int i1, int i2,
                                           double& val, double* grad) {
  // x: Gauss point i0 of the node row (y = i1, z = i2)
  const double* np = sN + nb + SY * i1 + SZ * i2;
  const double n0 = np[0], n1 = np[1], n2 = np[2];
  const double xv = fma(T.B[i0][2], n2, fma(T.B[i0][1], n1, T.B[i0][0] * n0));
  const double xd = GRAD ? fma(T.G[i0][2], n2, fma(T.G[i0][1], n1, T.G[i0][0] * n0)) : 0.0;
  // y: Gauss points (i0, i1) of node layer z = i2, from lanes (i0, a, i2)
  double yv = 0.0, ydy = 0.0, ydx = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int src = i0 + 3 * a + 9 * i2;
    const double v = __shfl_sync(FULL, xv, src);
    yv = fma(T.B[i1][a], v, yv);
    if (GRAD) {
      ydy = fma(T.G[i1][a], v, ydy);
      ydx = fma(T.B[i1][a], __shfl_sync(FULL, xd, src), ydx);
    }
  }
  // z: Gauss point (i0, i1, i2), from lanes (i0, i1, a)
  double v = 0.0, dx = 0.0, dy = 0.0, dz = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int src = i0 + 3 * i1 + 9 * a;
    const double w = __shfl_sync(FULL, yv, src);
    v = fma(T.B[i2][a], w, v);
    if (GRAD) {
      dz = fma(T.G[i2][a], w, dz);
      dx = fma(T.B[i2][a], __shfl_sync(FULL, ydx, src), dx);
      dy = fma(T.B[i2][a], __shfl_sync(FULL, ydy, src), dy);
    }
  }
  val = v;
  if (GRAD) {
    grad[0] = dx;
    grad[1] = dy;
    grad[2] = dz;
  }
}

// Test-side sum: lane (i0, i1, i2) returns sum_g w_g (s_g N_a(g) + f_g . grad N_a(g)) for local
// node a = (i0, i1, i2), from the Gauss-point integrands (s, f) held by lane g. DIAG: squared
// tables, the diagonal sum_g w_g (s_g N_a^2 + sum_d f_dg (dN_a/dx_d)^2). Warp-uniform call.
template <bool DIAG>
__device__ __forceinline__ double q2h_accum(const Q2HTab& T, double s, double fx, double fy, double fz, int i0, int i1,
                                            int i2) {
  const double(*BW)[3] = DIAG ? T.BB : T.BW;
  const double(*GW)[3] = DIAG ? T.GG : T.GW;
  // z: lane (gx = i0, gy = i1, node layer i2) from lanes (i0, i1, gz)
  double V = 0.0, X = 0.0, Y = 0.0;
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const int src = i0 + 3 * i1 + 9 * g;
    V = fma(BW[g][i2], __shfl_sync(FULL, s, src), V);
    V = fma(GW[g][i2], __shfl_sync(FULL, fz, src), V);
    X = fma(BW[g][i2], __shfl_sync(FULL, fx, src), X);
    Y = fma(BW[g][i2], __shfl_sync(FULL, fy, src), Y);
  }
  // y: lane (gx = i0, node row i1, layer i2) from lanes (i0, gy, i2)
  double V2 = 0.0, X2 = 0.0;
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const int src = i0 + 3 * g + 9 * i2;
    V2 = fma(BW[g][i1], __shfl_sync(FULL, V, src), V2);
    V2 = fma(GW[g][i1], __shfl_sync(FULL, Y, src), V2);
    X2 = fma(BW[g][i1], __shfl_sync(FULL, X, src), X2);
  }
  // x: node (i0, i1, i2) from lanes (gx, i1, i2)
  double r = 0.0;
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const int src = g + 3 * i1 + 9 * i2;
    r = fma(BW[g][i0], __shfl_sync(FULL, V2, src), r);
    r = fma(GW[g][i0], __shfl_sync(FULL, X2, src), r);
  }
  return r;
}

template <int MODEL, int MODE>
__global__ void __launch_bounds__(HTHREADS, 1) q2h_kernel(const Q2HArgs A) {
  constexpr int NC = NLin<3, MODEL>::VALUE;
  constexpr bool needU = MODE != M_JV && MODE != M_JTV;
  constexpr bool needV = MODE == M_JV || MODE == M_JTV || MODE == M_PREV_T;
  constexpr int NUF = needU ? 7 : 1;  // phi, u, phi - phi^n, u - u^n, phi^n, phihat_old, u^n
  constexpr int NVF = needV ? 2 : 1;
  __shared__ double sU[NUF * HNT];
  __shared__ double sV[NVF * HNT];
  __shared__ double sC[2 * 27 * HNE];
  __shared__ Q2HTab sT;
  // the next tile colour may start on free SMs now (it waits at the node sums)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  const DevMesh& m = A.m;
  const DevPhys& P = A.P;
  int b = blockIdx.x;
  const int bx = b % A.ctx;
  b /= A.ctx;
  const int by = b % A.cty;
  const int bz = b / A.cty;
  const int tile_x = 2 * bx + (A.color & 1);
  const int tile_y = 2 * by + ((A.color >> 1) & 1);
  const int tile_z = 2 * bz + ((A.color >> 2) & 1);
  const int ex0 = tile_x * HX, ey0 = tile_y * HY, ez0 = tile_z * HZ;
  const int nx0 = 2 * ex0, ny0 = 2 * ey0, nz0 = 2 * ez0;
  const bool tf1 = P.time_form != 0;

  // ---- 1. stage the tile's nodes and the tables ---------------------------------------
  if (threadIdx.x < 9) {
    const int g = threadIdx.x / 3, a = threadIdx.x % 3;
    sT.B[g][a] = A.T.B[g][a];
    sT.G[g][a] = A.T.G[g][a];
    sT.BW[g][a] = A.T.BW[g][a];
    sT.GW[g][a] = A.T.GW[g][a];
    sT.BB[g][a] = A.T.BB[g][a];
    sT.GG[g][a] = A.T.GG[g][a];
  }
  for (int s = threadIdx.x; s < HNT; s += HTHREADS) {
    const int lx = s % HNX, ly = (s / HNX) % HNY, lz = s / (HNX * HNY);
    const int gx = nx0 + lx, gy = ny0 + ly, gz = nz0 + lz;
    const bool ok = gx < m.nnx && gy < m.nny && gz < m.nnz;
    const i64 node = gx + (i64)m.nnx * (gy + (i64)m.nny * gz);
    if (needU) {
      double phi = 0.0, u = 0.0, phin = 0.0, un = 0.0, pho = 0.0;
      if (ok) {
        phi = A.U[node];
        u = A.U[m.nn + node];
        phin = A.Un[node];
        un = A.Un[m.nn + node];
        if (A.phold) pho = A.phold[node];
      }
      sU[0 * HNT + s] = phi;
      sU[1 * HNT + s] = u;
      sU[2 * HNT + s] = phi - phin;
      sU[3 * HNT + s] = u - un;
      sU[4 * HNT + s] = phin;
      sU[5 * HNT + s] = pho;
      sU[6 * HNT + s] = un;
    }
    if (needV) {
      sV[0 * HNT + s] = ok ? A.V[node] : 0.0;
      sV[1 * HNT + s] = ok ? A.V[m.nn + node] : 0.0;
    }
  }
  __syncthreads();

  // ---- 2./3. element arithmetic: warp e, lane l ---------------------------------------------
  const int e = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = lane < 27 ? lane : 26;
  const int i0 = l % 3, i1 = (l / 3) % 3, i2 = l / 9;
  const int lx = e % HX, ly = (e / HX) % HY, lz = e / (HX * HY);
  const int ex = ex0 + lx, ey = ey0 + ly, ez = ez0 + lz;
  const bool valid = ex < m.nx && ey < m.ny && ez < m.nz;  // uniform across the warp
  double r0 = 0.0, r1 = 0.0;
  if (valid) {
    const Q2HTab& T = sT;
    const int nb = 2 * lx + HNX * (2 * ly + HNY * 2 * lz);
    const i64 tile_id = tile_x + (i64)A.ntx * (tile_y + (i64)A.nty * tile_z);
    double* linp = A.lin + tile_id * (i64)(NC * HNE * 32) + e * 32 + lane;  // [c][element][lane]
    GPOut<3> o;
    if constexpr (MODE == M_JV || MODE == M_JTV) {
      double v0, v1, xp[3], xg[3];
      q2h_interp<true>(T, sV, nb, i0, i1, i2, v0, xp);
      q2h_interp<true>(T, sV + HNT, nb, i0, i1, i2, v1, xg);
      double L[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) L[c] = __ldg(linp + c * HNE * 32);
      lin_apply<3, MODEL, MODE == M_JTV>(P, L, v0, v1, xp, xg, o);
    } else {
      double phi, u, dphi, du, p[3], gg[3];
      q2h_interp<true>(T, sU, nb, i0, i1, i2, phi, p);
      q2h_interp<true>(T, sU + HNT, nb, i0, i1, i2, u, gg);
      q2h_interp<false>(T, sU + 2 * HNT, nb, i0, i1, i2, dphi, nullptr);
      q2h_interp<false>(T, sU + 3 * HNT, nb, i0, i1, i2, du, nullptr);
      // grad(phi^n): literal time term; level-n flux of the theta-method in the adjoint modes
      const bool oldn = (MODE == M_DEPS || MODE == M_PREV_T) && P.theta != 1.0;
      double pn[3] = {0.0, 0.0, 0.0};
      if ((tf1 || oldn) && MODE != M_OLD && MODE != M_DIAG) {
        double pnv;
        q2h_interp<true>(T, sU + 4 * HNT, nb, i0, i1, i2, pnv, pn);
      }
      double pho = 0.0;
      if ((MODE == M_RES || MODE == M_RES_LIN) && P.phihat_old)
        q2h_interp<false>(T, sU + 5 * HNT, nb, i0, i1, i2, pho, nullptr);
      double G4 = 0.0, G4n = 0.0;
      if (MODEL == 1 && P.has_g4) {
        const double z = fma(m.h, ez + A.T.xg[i2], m.z0);
        G4 = (z - P.zT - P.Vp * (MODE == M_OLD ? P.t_new - P.dt : P.t_new)) / P.lT;
        G4n = (z - P.zT - P.Vp * (P.t_new - P.dt)) / P.lT;
      }
      if (MODE == M_DIAG) {
        // Eqs. (pref2), (preconc2) at the Gauss point: mass and stiffness coefficients of M11, M22
        Aniso<3> An;
        An.eval(p, P.eps4);
        const double a2 = An.a * An.a;
        const double B = fma(1.0 - P.k, u, 1.0);
        const double phin = phi - dphi;
        const double Acoef = MODEL == 0 ? 1.0 : 0.5 * ((1.0 + P.k) - (1.0 - P.k) * phin);
        const double q = MODEL == 0 ? 1.0 : 0.5 * (1.0 - phi);
        o.sphi = P.tau0 * B * a2 * P.idt;
        o.fphi[0] = o.fphi[1] = o.fphi[2] = P.thW2 * a2;
        o.su = Acoef * P.idt;
        o.fu[0] = o.fu[1] = o.fu[2] = P.thD * q;
      } else if (MODE == M_OLD) {
        spatial_old<3, MODEL>(P, phi, u, p, gg, G4, o);
      } else if (MODE == M_RES || MODE == M_RES_LIN) {
        double L[MODE == M_RES_LIN ? NC : 1];
        pointwise<3, MODEL, MODE == M_RES_LIN>(P, A.C, phi, u, dphi, du, pho, p, gg, pn, G4, o, L, A.Ku);
        if (MODE == M_RES_LIN && lane < 27) {
#pragma unroll
          for (int c = 0; c < NC; ++c) linp[c * HNE * 32] = L[c];
        }
      } else if (MODE == M_DEPS) {
        gp_deps<3>(P, tf1, phi, u, dphi, du, p, pn, o);
      } else {  // M_PREV_T
        double w0, w1, gw0[3], gw1[3];
        q2h_interp<true>(T, sV, nb, i0, i1, i2, w0, gw0);
        q2h_interp<true>(T, sV + HNT, nb, i0, i1, i2, w1, gw1);
        double unv = 0.0, gn[3] = {0.0, 0.0, 0.0};
        if (oldn) q2h_interp<true>(T, sU + 6 * HNT, nb, i0, i1, i2, unv, gn);
        gp_prev_t<3, MODEL>(P, tf1, phi, u, dphi, du, p, pn, w0, w1, gw1, o);
        if (oldn) old_spatial_t<3, MODEL>(P, phi - dphi, u - du, pn, gn, G4n, w0, gw0, gw1, o);
      }
    }
    r0 = q2h_accum<MODE == M_DIAG>(T, o.sphi, o.fphi[0], o.fphi[1], o.fphi[2], i0, i1, i2);
    r1 = q2h_accum<MODE == M_DIAG>(T, o.su, o.fu[0], o.fu[1], o.fu[2], i0, i1, i2);
  }
  if (lane < 27) {
    sC[lane * HNE + e] = r0;
    sC[(27 + lane) * HNE + e] = r1;
  }
  __syncthreads();

  // ---- 4. node sums in fixed order, read-modify-write ---------------------------------------
  // a colour launched as a programmatic dependent of the previous one waits here for that
  // grid's node sums (a no-op after an ordinary launch); the reads bypass L1
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int s = threadIdx.x; s < HNT; s += HTHREADS) {
    const int nxl = s % HNX, nyl = (s / HNX) % HNY, nzl = s / (HNX * HNY);
    const int gx = nx0 + nxl, gy = ny0 + nyl, gz = nz0 + nzl;
    if (gx >= m.nnx || gy >= m.nny || gz >= m.nnz) continue;
    double acc0 = 0.0, acc1 = 0.0;
    // along each axis a node is local node 2 of element i/2 - 1 and local node 0 of
    // element i/2 (i even), or local node 1 of element (i - 1)/2 (i odd)
#pragma unroll
    for (int cz = 0; cz < 2; ++cz) {
      const int elz = (nzl & 1) ? (cz == 0 ? (nzl - 1) / 2 : -1) : nzl / 2 - 1 + cz;
      const int az = (nzl & 1) ? 1 : 2 - 2 * cz;
#pragma unroll
      for (int cy = 0; cy < 2; ++cy) {
        const int ely = (nyl & 1) ? (cy == 0 ? (nyl - 1) / 2 : -1) : nyl / 2 - 1 + cy;
        const int ay = (nyl & 1) ? 1 : 2 - 2 * cy;
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
          const int elx = (nxl & 1) ? (cx == 0 ? (nxl - 1) / 2 : -1) : nxl / 2 - 1 + cx;
          const int ax = (nxl & 1) ? 1 : 2 - 2 * cx;
          if (elx >= 0 && elx < HX && ely >= 0 && ely < HY && elz >= 0 && elz < HZ) {
            const int el = elx + HX * (ely + HY * elz);
            const int a = ax + 3 * (ay + 3 * az);
            acc0 += sC[a * HNE + el];
            acc1 += sC[(27 + a) * HNE + el];
          }
        }
      }
    }
    const i64 node = gx + (i64)m.nnx * (gy + (i64)m.nny * gz);
    A.out[node] = __ldcg(A.out + node) + acc0;
    A.out[m.nn + node] = __ldcg(A.out + m.nn + node) + acc1;
  }
}

template <int MODEL, int MODE>
static cudaError_t q2h_colours(const ElemCtx& c, Q2HArgs a, cudaStream_t st) {
  for (int col = 0; col < 8; ++col) {
    const int cx = col & 1, cy = (col >> 1) & 1, cz = (col >> 2) & 1;
    a.color = col;
    a.ctx = (c.ntx - cx + 1) / 2;
    a.cty = (c.nty - cy + 1) / 2;
    a.ctz = (c.ntz - cz + 1) / 2;
    const long long blocks = (long long)a.ctx * a.cty * a.ctz;
    if (blocks <= 0) continue;
    const cudaError_t e = launch_colour(q2h_kernel<MODEL, MODE>, (unsigned)blocks, HTHREADS, 0, st, col > 0, a);
    if (e != cudaSuccess) return e;
    count_launches(1);
  }
  return cudaGetLastError();
}

template <int MODEL>
static cudaError_t q2h_dispatch(int mode, const ElemCtx& c, const Q2HArgs& a, cudaStream_t st) {
  switch (mode) {
    case M_RES: return q2h_colours<MODEL, M_RES>(c, a, st);
    case M_RES_LIN: return q2h_colours<MODEL, M_RES_LIN>(c, a, st);
    case M_JV: return q2h_colours<MODEL, M_JV>(c, a, st);
    case M_JTV: return q2h_colours<MODEL, M_JTV>(c, a, st);
    case M_DEPS: return q2h_colours<MODEL, M_DEPS>(c, a, st);
    case M_PREV_T: return q2h_colours<MODEL, M_PREV_T>(c, a, st);
    case M_OLD: return q2h_colours<MODEL, M_OLD>(c, a, st);
    case M_DIAG: return q2h_colours<MODEL, M_DIAG>(c, a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t q2h_run(int mode, const ElemCtx& c, const double* U, const double* Un, const double* V, double* out,
                    double* lin, cudaStream_t st, const double* phold) {
  if (c.m.dim != 3 || c.m.order != 2) return cudaErrorInvalidValue;
  Q2HArgs a;
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
  a.nty = c.nty;
  a.color = 0;
  a.ctx = a.cty = a.ctz = 0;
  return c.P.model == 0 ? q2h_dispatch<0>(mode, c, a, st) : q2h_dispatch<1>(mode, c, a, st);
}


// ---------------------------------------------------------------------------
// Preconditioner blocks M11, M22 (Eqs. pref2, preconc2) of a triquadratic box for
// the multigrid: 125-point stencils [2][125][nn] on its node lattice (spacing h/2),
// and 27-point stencils [2][27][nv] on the grid of element vertices. The vertex
// level is P^T A P for the trilinear prolongation, which embeds the trilinear space
// of each element exactly in its triquadratic one, so it is built directly as the
// trilinear element matrices with the same 27 Gauss-point coefficients (the
// Galerkin product without the 125 x 27 contraction). One warp per element, lanes =
// Gauss points for the coefficients, then lane a sums row a of the element matrix
// (and lanes 0..7 the trilinear rows) and adds it to the stencil rows of its node.
// Elements run in 8 colours (index parity per axis): elements of one colour share no
// node, so the read-modify-writes of a launch never collide, and the colours run in
// a fixed order (deterministic). Arithmetic of the sums in the stencil precision T.
// ---------------------------------------------------------------------------
template <typename T>
struct Q2HFillArgs {
  DevMesh m;   // the Q2 mesh
  DevPhys P;
  Q2Tab Tb;
  const double* U;
  const double* Un;
  T* st;       // lattice stencils [2][125][nn], zeroed before the first colour
  T* stv;      // vertex-grid stencils [2][27][nv], zeroed, or null
  int nvx, nvy;  // vertex grid nodes per axis (nx + 1, ny + 1)
  i64 nv;
  int color;
  int ncx, ncy;  // elements of this colour per axis (x, y)
  int ncol;      // elements of this colour
};

template <int MODEL, typename T>
__global__ void __launch_bounds__(128) k_q2h_stencil_fill(const Q2HFillArgs<T> A) {
  constexpr int W = 4;  // warps (elements) per CTA
  __shared__ Q2HTab sT;
  __shared__ T sN[27][27], sGx[27][27], sGy[27][27], sGz[27][27];  // [g][b] Q2 basis, physical gradient
  __shared__ T sN1[27][8], sG1x[27][8], sG1y[27][8], sG1z[27][8];  // trilinear basis of the vertices
  __shared__ double sNod[W][3][27];                                 // phi, u, phi^n of the element nodes
  __shared__ T sC[W][4][27];                                         // weighted coefficients per Gauss point
  const DevMesh& m = A.m;
  const DevPhys& P = A.P;
  for (int t = threadIdx.x; t < 27 * 27; t += blockDim.x) {
    const int g = t / 27, b = t % 27;
    const int gx = g % 3, gy = (g / 3) % 3, gz = g / 9, bx = b % 3, by = (b / 3) % 3, bz = b / 9;
    const Q2Tab& Q = A.Tb;
    sN[g][b] = T(Q.B[gx][bx] * Q.B[gy][by] * Q.B[gz][bz]);
    sGx[g][b] = T(Q.G[gx][bx] * Q.B[gy][by] * Q.B[gz][bz]);
    sGy[g][b] = T(Q.B[gx][bx] * Q.G[gy][by] * Q.B[gz][bz]);
    sGz[g][b] = T(Q.B[gx][bx] * Q.B[gy][by] * Q.G[gz][bz]);
    if (b < 8) {
      const int vx = b & 1, vy = (b >> 1) & 1, vz = b >> 2;
      const double xs[3] = {Q.xg[gx], Q.xg[gy], Q.xg[gz]};
      const int v[3] = {vx, vy, vz};
      double l[3], dl[3];
      for (int d = 0; d < 3; ++d) {
        l[d] = v[d] ? xs[d] : 1.0 - xs[d];
        dl[d] = (v[d] ? 1.0 : -1.0) / m.h;
      }
      sN1[g][b] = T(l[0] * l[1] * l[2]);
      sG1x[g][b] = T(dl[0] * l[1] * l[2]);
      sG1y[g][b] = T(l[0] * dl[1] * l[2]);
      sG1z[g][b] = T(l[0] * l[1] * dl[2]);
    }
  }
  if (threadIdx.x < 9) {
    const int g = threadIdx.x / 3, a = threadIdx.x % 3;
    sT.B[g][a] = A.Tb.B[g][a];
    sT.G[g][a] = A.Tb.G[g][a];
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = lane < 27 ? lane : 26;
  const int i0 = l % 3, i1 = (l / 3) % 3, i2 = l / 9;
  const int eid = blockIdx.x * W + w;
  const bool valid = eid < A.ncol;  // uniform across the warp
  const int ci = valid ? eid % A.ncx : 0, cj = valid ? (eid / A.ncx) % A.ncy : 0,
            ck = valid ? eid / (A.ncx * A.ncy) : 0;
  const int ex = 2 * ci + (A.color & 1), ey = 2 * cj + ((A.color >> 1) & 1), ez = 2 * ck + ((A.color >> 2) & 1);
  const i64 node = (2 * ex + i0) + (i64)m.nnx * ((2 * ey + i1) + (i64)m.nny * (2 * ez + i2));
  if (valid && lane < 27) {
    sNod[w][0][lane] = A.U[node];
    sNod[w][1][lane] = A.U[m.nn + node];
    sNod[w][2][lane] = A.Un[node];
  }
  __syncthreads();
  if (!valid) return;
  // Gauss-point coefficients (lane = Gauss point), weights included
  {
    double phi, u, phin, p[3], gu[3];
    q2h_interp<true, 3, 9>(sT, &sNod[w][0][0], 0, i0, i1, i2, phi, p);
    q2h_interp<false, 3, 9>(sT, &sNod[w][1][0], 0, i0, i1, i2, u, gu);
    q2h_interp<false, 3, 9>(sT, &sNod[w][2][0], 0, i0, i1, i2, phin, nullptr);
    Aniso<3> An;
    An.eval(p, P.eps4);
    const double a2 = An.a * An.a;
    const double B = fma(1.0 - P.k, u, 1.0);
    const double Acoef = MODEL == 0 ? 1.0 : 0.5 * ((1.0 + P.k) - (1.0 - P.k) * phin);
    const double q = MODEL == 0 ? 1.0 : 0.5 * (1.0 - phi);
    const double wg = (5.0 + 3.0 * (i0 == 1)) * (5.0 + 3.0 * (i1 == 1)) * (5.0 + 3.0 * (i2 == 1)) / 5832.0 *
                      m.h * m.h * m.h;  // (5/18 or 8/18)^3 h^3
    if (lane < 27) {
      sC[w][0][lane] = T(wg * P.tau0 * B * a2 * P.idt);
      sC[w][1][lane] = T(wg * P.thW2 * a2);
      sC[w][2][lane] = T(wg * Acoef * P.idt);
      sC[w][3][lane] = T(wg * P.thD * q);
    }
  }
  __syncwarp();
  // row a = lane of the triquadratic element matrices of both blocks
  if (lane < 27) {
    const int a = lane;
    T acc0[27], acc1[27];
#pragma unroll
    for (int b = 0; b < 27; ++b) acc0[b] = acc1[b] = T(0);
#pragma unroll 1
    for (int g = 0; g < 27; ++g) {
      const T na = sN[g][a], xa = sGx[g][a], ya = sGy[g][a], za = sGz[g][a];
      const T m0 = sC[w][0][g] * na, k0 = sC[w][1][g], m1 = sC[w][2][g] * na, k1 = sC[w][3][g];
      const T k0x = k0 * xa, k0y = k0 * ya, k0z = k0 * za, k1x = k1 * xa, k1y = k1 * ya, k1z = k1 * za;
#pragma unroll
      for (int b = 0; b < 27; ++b) {
        const T nb = sN[g][b], xb = sGx[g][b], yb = sGy[g][b], zb = sGz[g][b];
        acc0[b] += m0 * nb + k0x * xb + k0y * yb + k0z * zb;
        acc1[b] += m1 * nb + k1x * xb + k1y * yb + k1z * zb;
      }
    }
#pragma unroll
    for (int b = 0; b < 27; ++b) {
      const int o = (b % 3 - i0 + 2) + 5 * ((b / 3) % 3 - i1 + 2) + 25 * (b / 9 - i2 + 2);
      A.st[(i64)o * m.nn + node] += acc0[b];
      A.st[(i64)(125 + o) * m.nn + node] += acc1[b];
    }
  }
  // vertex rows of the trilinear element matrices (lanes 0..7)
  if (A.stv && lane < 8) {
    const int vx = lane & 1, vy = (lane >> 1) & 1, vz = lane >> 2;
    T acc0[8], acc1[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) acc0[b] = acc1[b] = T(0);
#pragma unroll 1
    for (int g = 0; g < 27; ++g) {
      const T na = sN1[g][lane], xa = sG1x[g][lane], ya = sG1y[g][lane], za = sG1z[g][lane];
      const T m0 = sC[w][0][g] * na, k0 = sC[w][1][g], m1 = sC[w][2][g] * na, k1 = sC[w][3][g];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const T gd = xa * sG1x[g][b] + ya * sG1y[g][b] + za * sG1z[g][b];
        acc0[b] += m0 * sN1[g][b] + k0 * gd;
        acc1[b] += m1 * sN1[g][b] + k1 * gd;
      }
    }
    const i64 vnode = (ex + vx) + (i64)A.nvx * ((ey + vy) + (i64)A.nvy * (ez + vz));
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int o = ((b & 1) - vx + 1) + 3 * (((b >> 1) & 1) - vy + 1) + 9 * ((b >> 2) - vz + 1);
      A.stv[(i64)o * A.nv + vnode] += acc0[b];
      A.stv[(i64)(27 + o) * A.nv + vnode] += acc1[b];
    }
  }
}

template <typename T>
cudaError_t q2h_stencil_fill(const ElemCtx& c, const double* U, const double* Un, T* st, T* stv, cudaStream_t s) {
  const DevMesh& m = c.m;
  if (m.dim != 3 || m.order != 2) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(T) * 2 * 125 * (size_t)m.nn, s);
  if (e != cudaSuccess) return e;
  Q2HFillArgs<T> a;
  a.m = m;
  a.P = c.P;
  a.Tb = c.q2;
  a.U = U;
  a.Un = Un;
  a.st = st;
  a.stv = stv;
  a.nvx = m.nx + 1;
  a.nvy = m.ny + 1;
  a.nv = (i64)(m.nx + 1) * (m.ny + 1) * (m.nz + 1);
  if (stv) {
    e = cudaMemsetAsync(stv, 0, sizeof(T) * 2 * 27 * (size_t)a.nv, s);
    if (e != cudaSuccess) return e;
  }
  for (int col = 0; col < 8; ++col) {
    const int cx = col & 1, cy = (col >> 1) & 1, cz = (col >> 2) & 1;
    a.color = col;
    a.ncx = (m.nx - cx + 1) / 2;
    a.ncy = (m.ny - cy + 1) / 2;
    const int ncz = (m.nz - cz + 1) / 2;
    a.ncol = a.ncx * a.ncy * ncz;
    if (a.ncol <= 0) continue;
    const int blocks = (a.ncol + 3) / 4;
    if (c.P.model == 0)
      k_q2h_stencil_fill<0, T><<<blocks, 128, 0, s>>>(a);
    else
      k_q2h_stencil_fill<1, T><<<blocks, 128, 0, s>>>(a);
    count_launches(1);
  }
  return cudaGetLastError();
}
template cudaError_t q2h_stencil_fill<float>(const ElemCtx&, const double*, const double*, float*, float*,
                                             cudaStream_t);
template cudaError_t q2h_stencil_fill<double>(const ElemCtx&, const double*, const double*, double*, double*,
                                              cudaStream_t);

}  // namespace tusas
