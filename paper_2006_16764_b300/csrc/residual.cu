// Element-tile kernels: residual F(U), residual + pointwise linearisation,
// stored-linearisation tangent J v and adjoint J^T w, dF/d eps4 and
// (dF/dU^n)^T w, on structured Q1 boxes (Sec. 2.1.1, Sec. 4.2).
//
// Data path of one CTA (one tile of Tile<DIM> elements, one thread per element):
//   1. the tile's (T+1)^dim nodes of the needed fields are staged in shared
//      memory with coalesced loads along x;
//   2. each thread interpolates its element's fields to the 2^dim Gauss points
//      (sum factorisation, element.cuh), evaluates the pointwise integrands in
//      registers and accumulates the 2 x 2^dim nodal contributions;
//   3. contributions go to shared memory and each tile node sums its <= 2^dim
//      element contributions in a fixed order, then adds the sum to the global
//      vector (read-modify-write).
// Tiles are launched in 2^dim colours (parity of the tile index per axis), so
// tiles that run concurrently never share a node: no atomics, and the result
// is bitwise reproducible (the paper's element colouring, Sec. 4.3, lifted to
// tiles).
#include "ops.h"

namespace tusas {

struct ElemArgs {
  DevMesh m;
  DevPhys P;
  double h, inv_h;  // element size and its inverse
  double wh;        // Gauss weight over h, w / h: the node-sum factor of the residual-type passes
  LinScale K;       // staged-form linearisation factors (tangent / adjoint passes)
  PwConst C;        // pointwise constants for the gradient units of the kernel (true, or staged in 3D)
  const double* U;
  const double* Un;
  const double* V;
  double* out;
  double* lin;
  const double* phold;  // nodal (phi^n - phi^{n-1})/dt for the Eq. (theta) estimate, or null
  int color;
  int ctx, cty, ctz;  // tiles of this colour per axis
  int ntx, nty;       // tiles per axis (for the tile id)
};

template <int DIM>
__device__ __forceinline__ double gp_last_coord(const DevMesh& m, int e_last, int g) {
  const double s = 0.57735026918962576;
  const double org = DIM == 3 ? m.z0 : m.y0;
  const double off = ((g >> (DIM - 1)) & 1) ? 0.5 * (1.0 + s) : 0.5 * (1.0 - s);
  return org + m.h * (e_last + off);
}

template <int MODE>
struct MinBlocks {
  static const int V = MODE == 2 || MODE == 3 ? 3 : 2;  // tangent and adjoint: 3 CTAs / SM (no spills)
};

template <int DIM, int MODEL, int MODE>
__global__ void __launch_bounds__(Tile<DIM>::X * Tile<DIM>::Y * Tile<DIM>::Z, MinBlocks<MODE>::V)
elem_kernel(const ElemArgs A) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  constexpr int NX = TX + 1, NY = TY + 1, NZ = DIM == 3 ? TZ + 1 : 1;
  constexpr int NT = NX * NY * NZ;
  constexpr int NE = TX * TY * TZ;
  constexpr int NN = 1 << DIM;
  constexpr int NH = NN / 2;
  constexpr int NC = NLin<DIM, MODEL>::VALUE;
  constexpr bool needU = MODE != M_JV && MODE != M_JTV;
  constexpr bool needV = MODE == M_JV || MODE == M_JTV || MODE == M_PREV_T;
  constexpr int NUF = needU ? 6 : 1;
  constexpr int NVF = needV ? 2 : 1;

  __shared__ double sU[NUF][NT];  // phi, u, phi - phi^n, u - u^n, phi^n, phihat_old
  __shared__ double sV[NVF][NT];
  __shared__ double sC[2 * NN][NE];

  // the next tile colour may start on free SMs now (it waits at the node sums)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const DevMesh& m = A.m;
  int b = blockIdx.x;
  const int ix = b % A.ctx;
  b /= A.ctx;
  const int iy = b % A.cty;
  const int iz = b / A.cty;
  const int tile_x = 2 * ix + (A.color & 1);
  const int tile_y = 2 * iy + ((A.color >> 1) & 1);
  const int tile_z = DIM == 3 ? 2 * iz + ((A.color >> 2) & 1) : 0;
  const int ex0 = tile_x * TX, ey0 = tile_y * TY, ez0 = tile_z * TZ;
  const bool tf1 = A.P.time_form != 0;

  // ---- 1. stage the tile's nodes --------------------------------------------
  for (int s = threadIdx.x; s < NT; s += NE) {
    const int lx = s % NX, ly = (s / NX) % NY, lz = s / (NX * NY);
    const int gx = ex0 + lx, gy = ey0 + ly, gz = ez0 + lz;
    const bool ok = gx < m.nnx && gy < m.nny && gz < m.nnz;
    const i64 node = gx + (i64)m.nnx * (gy + (i64)m.nny * gz);
    if (needU) {
      double phi = 0.0, u = 0.0, phin = 0.0, un = 0.0;
      if (ok) {
        phi = A.U[node];
        u = A.U[m.nn + node];
        phin = A.Un[node];
        un = A.Un[m.nn + node];
      }
      sU[0][s] = phi;
      sU[1][s] = u;
      sU[2][s] = phi - phin;
      sU[3][s] = u - un;
      sU[4][s] = phin;
      sU[NUF - 1][s] = (A.phold && ok) ? A.phold[node] : 0.0;
    }
    if (needV) {
      sV[0][s] = ok ? A.V[node] : 0.0;
      sV[NVF - 1][s] = ok ? A.V[m.nn + node] : 0.0;
    }
  }
  __syncthreads();

  // ---- 2. element arithmetic --------------------------------------------------
  const int t = threadIdx.x;
  const int lx = t % TX, ly = (t / TX) % TY, lz = t / (TX * TY);
  const int ex = ex0 + lx, ey = ey0 + ly, ez = ez0 + lz;
  const bool valid = ex < m.nx && ey < m.ny && (DIM == 2 || ez < m.nz);
  double r0[NN], r1[NN];
#pragma unroll
  for (int a = 0; a < NN; ++a) r0[a] = r1[a] = 0.0;
  if (valid) {
    int sidx[NN];
#pragma unroll
    for (int a = 0; a < NN; ++a) sidx[a] = (lx + (a & 1)) + NX * ((ly + ((a >> 1) & 1)) + NY * (lz + ((a >> 2) & 1)));
    const i64 tile_id = tile_x + (i64)A.ntx * (tile_y + (i64)A.nty * tile_z);
    double* linp = A.lin + tile_id * (i64)(NC * NN * NE) + t;  // [c][g][t] within the tile
    GPOut<DIM> o;
    double s0[NN], s1[NN], f0[DIM][NN], f1[DIM][NN];
    if (MODE == M_JV || MODE == M_JTV) {
      double v0[NN], v1[NN], gv0[DIM][NH], gv1[DIM][NH], n0[NN], n1[NN];
#pragma unroll
      for (int a = 0; a < NN; ++a) {
        n0[a] = sV[0][sidx[a]];
        n1[a] = sV[NVF - 1][sidx[a]];
      }
      interp_l<DIM>(n0, v0, gv0);
      interp_l<DIM>(n1, v1, gv1);
#pragma unroll
      for (int g = 0; g < NN; ++g) {
        double L[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) L[c] = __ldg(linp + (c * NN + g) * NE);
        double xp[DIM], xg[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          xp[d] = gv0[d][remove_bit(g, d)];
          xg[d] = gv1[d][remove_bit(g, d)];
        }
        lin_apply<DIM, MODEL, MODE == M_JTV, true>(A.P, L, v0[g], v1[g], xp, xg, o, A.K);
        s0[g] = o.sphi;
        s1[g] = o.su;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          f0[d][g] = o.fphi[d];
          f1[d][g] = o.fu[d];
        }
      }
    } else {
      double nphi[NN], nu[NN], ndp[NN], ndu[NN];
#pragma unroll
      for (int a = 0; a < NN; ++a) {
        nphi[a] = sU[0][sidx[a]];
        nu[a] = sU[1][sidx[a]];
        ndp[a] = sU[2][sidx[a]];
        ndu[a] = sU[3][sidx[a]];
      }
      double phi[NN], u[NN], dphi[NN], du[NN], gp[DIM][NH], gu[DIM][NH], gpn[DIM][NH];
      interp_true<DIM, true>(nphi, phi, gp, A.inv_h);
      interp_true<DIM, true>(nu, u, gu, A.inv_h);
      interp_true<DIM, false>(ndp, dphi, nullptr, A.inv_h);
      interp_true<DIM, false>(ndu, du, nullptr, A.inv_h);
      // grad(phi^n): literal time term, or the level-n flux of the theta-method in dF/d eps4 and
      // (dF/dU^n)^T w; grad(u^n) for the latter
      const bool oldn = (MODE == M_DEPS || MODE == M_PREV_T) && A.P.theta != 1.0;
      double gun[DIM][NH];
      if (tf1 || oldn) {
        double npn[NN], vpn[NN];
#pragma unroll
        for (int a = 0; a < NN; ++a) npn[a] = sU[4][sidx[a]];
        interp_true<DIM, true>(npn, vpn, gpn, A.inv_h);
      }
      if (MODE == M_PREV_T && oldn) {
        double nun[NN], vun[NN];
#pragma unroll
        for (int a = 0; a < NN; ++a) nun[a] = sU[1][sidx[a]] - sU[3][sidx[a]];
        interp_true<DIM, true>(nun, vun, gun, A.inv_h);
      }
      double pho[NN];
      if ((MODE == M_RES || MODE == M_RES_LIN) && A.P.phihat_old) {
        double npo[NN];
#pragma unroll
        for (int a = 0; a < NN; ++a) npo[a] = sU[NUF - 1][sidx[a]];
        interp_true<DIM, false>(npo, pho, nullptr, A.inv_h);
      } else {
#pragma unroll
        for (int a = 0; a < NN; ++a) pho[a] = 0.0;
      }
      double w0[NN], w1[NN], gw0[DIM][NH], gw1[DIM][NH];
      if (MODE == M_PREV_T) {
        double n0[NN], n1[NN];
#pragma unroll
        for (int a = 0; a < NN; ++a) {
          n0[a] = sV[0][sidx[a]];
          n1[a] = sV[NVF - 1][sidx[a]];
        }
        interp_true<DIM, true>(n0, w0, gw0, A.inv_h);
        interp_true<DIM, true>(n1, w1, gw1, A.inv_h);
      }
      const int e_last = DIM == 3 ? ez : ey;
#pragma unroll
      for (int g = 0; g < NN; ++g) {
        double p[DIM], gg[DIM], pn[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          p[d] = gp[d][remove_bit(g, d)];
          gg[d] = gu[d][remove_bit(g, d)];
          pn[d] = (tf1 || oldn) ? gpn[d][remove_bit(g, d)] : 0.0;
        }
        double G4 = 0.0;
        if (MODEL == 1 && A.P.has_g4) {
          const double tl = MODE == M_OLD ? A.P.t_new - A.P.dt : A.P.t_new;
          G4 = (gp_last_coord<DIM>(m, e_last, g) - A.P.zT - A.P.Vp * tl) / A.P.lT;
        }
        if (MODE == M_OLD) {
          spatial_old<DIM, MODEL>(A.P, phi[g], u[g], p, gg, G4, o);
        } else if (MODE == M_RES || MODE == M_RES_LIN) {
          double L[MODE == M_RES_LIN ? NC : 1];
          pointwise<DIM, MODEL, MODE == M_RES_LIN>(A.P, A.C, phi[g], u[g], dphi[g], du[g], pho[g], p, gg, pn, G4, o,
                                                   L, A.K);
          if (MODE == M_RES_LIN) {
#pragma unroll
            for (int c = 0; c < NC; ++c) linp[(c * NN + g) * NE] = L[c];
          }
        } else if (MODE == M_DEPS) {
          gp_deps<DIM>(A.P, tf1, phi[g], u[g], dphi[g], du[g], p, pn, o);
        } else {  // M_PREV_T
          double gw[DIM];
#pragma unroll
          for (int d = 0; d < DIM; ++d) gw[d] = gw1[d][remove_bit(g, d)];
          gp_prev_t<DIM, MODEL>(A.P, tf1, phi[g], u[g], dphi[g], du[g], p, pn, w0[g], w1[g], gw, o);
          if (oldn) {
            double gn[DIM], gv0[DIM];
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
              gn[d] = gun[d][remove_bit(g, d)];
              gv0[d] = gw0[d][remove_bit(g, d)];
            }
            const double G4n = (MODEL == 1 && A.P.has_g4)
                                   ? (gp_last_coord<DIM>(m, e_last, g) - A.P.zT - A.P.Vp * (A.P.t_new - A.P.dt)) / A.P.lT
                                   : 0.0;
            old_spatial_t<DIM, MODEL>(A.P, phi[g] - dphi[g], u[g] - du[g], pn, gn, G4n, w0[g], gv0, gw, o);
          }
        }
        // true-unit integrands: values times h here, the node sums times w / h
        s0[g] = o.sphi * A.h;
        s1[g] = o.su * A.h;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          f0[d][g] = o.fphi[d];
          f1[d][g] = o.fu[d];
        }
      }
    }
    accumulate_l<DIM>(s0, f0, r0);
    accumulate_l<DIM>(s1, f1, r1);
  }
#pragma unroll
  for (int a = 0; a < NN; ++a) {
    sC[a][t] = r0[a];
    sC[NN + a][t] = r1[a];
  }
  __syncthreads();

  // ---- 3. node sums in fixed order, read-modify-write ---------------------------
  // a colour launched as a programmatic dependent of the previous one waits here for that
  // grid's node sums (a no-op after an ordinary launch); the reads bypass L1
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int s = threadIdx.x; s < NT; s += NE) {
    const int nx_ = s % NX, ny_ = (s / NX) % NY, nz_ = s / (NX * NY);
    const int gx = ex0 + nx_, gy = ey0 + ny_, gz = ez0 + nz_;
    if (gx >= m.nnx || gy >= m.nny || gz >= m.nnz) continue;
    double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      const int elx = nx_ - (a & 1), ely = ny_ - ((a >> 1) & 1), elz = nz_ - ((a >> 2) & 1);
      if (elx >= 0 && elx < TX && ely >= 0 && ely < TY && elz >= 0 && elz < TZ) {
        const int e = elx + TX * (ely + TY * elz);
        acc0 += sC[a][e];
        acc1 += sC[NN + a][e];
      }
    }
    if (MODE != M_JV && MODE != M_JTV) {
      acc0 *= A.wh;
      acc1 *= A.wh;
    }
    const i64 node = gx + (i64)m.nnx * (gy + (i64)m.nny * gz);
    A.out[node] = __ldcg(A.out + node) + acc0;
    A.out[m.nn + node] = __ldcg(A.out + m.nn + node) + acc1;
  }
}

#include "tile3.cuh"

void elem_ctx_init(ElemCtx& c, const DevMesh& m, const DevPhys& P) {
  c.m = m;
  c.P = P;
  const int dim = m.dim;
  const double s = 1.0 / sqrt(3.0);
  const double nnodes = dim == 3 ? 8.0 : 4.0;
  const double w = dim == 3 ? (m.h / 2) * (m.h / 2) * (m.h / 2) : (m.h / 2) * (m.h / 2);
  for (int k = 0; k < 4; ++k) {
    c.S.vs[k] = pow(s, k) / nnodes;
    c.S.vsw[k] = c.S.vs[k] * w;
  }
  for (int k = 0; k < 3; ++k) {
    c.S.gs[k] = pow(s, k) * 2.0 / (m.h * nnodes);
    c.S.gsw[k] = c.S.gs[k] * w;
  }
  // staged forms: interp_l gives values and h times the gradients; accumulate_l takes
  // values times w and fluxes times w / h
  c.K.vv = w;
  c.K.gv = w / m.h;
  c.K.vf = w / m.h;
  c.K.gf = w / (m.h * m.h);
  lin_consts(c.K, P);
  c.Ku = lin_unit(P);
  c.pw_elem = pw_consts(P, c.K, 1.0);       // elem_kernel: true gradients, staged linearisation
  c.pw_res3 = pw_consts(P, c.K, 1.0 / m.h);  // res3_kernel: staged gradients and linearisation
  c.pw_q2 = pw_consts(P, c.Ku, 1.0);         // Q2 kernels: true units throughout
  if (dim == 3 && m.order == 2) {
    c.ntx = ceil_div(m.nx, Q2HexTile::X);
    c.nty = ceil_div(m.ny, Q2HexTile::Y);
    c.ntz = ceil_div(m.nz, Q2HexTile::Z);
    c.nlin = P.model == 0 ? NLin<3, 0>::VALUE : NLin<3, 1>::VALUE;
  } else if (dim == 3) {
    c.ntx = ceil_div(m.nx, Tile<3>::X);
    c.nty = ceil_div(m.ny, Tile<3>::Y);
    c.ntz = ceil_div(m.nz, Tile<3>::Z);
    c.nlin = P.model == 0 ? NLin<3, 0>::VALUE : NLin<3, 1>::VALUE;
  } else {
    c.ntx = ceil_div(m.nx, Tile<2>::X);
    c.nty = ceil_div(m.ny, Tile<2>::Y);
    c.ntz = 1;
    c.nlin = P.model == 0 ? NLin<2, 0>::VALUE : NLin<2, 1>::VALUE;
  }
  if (m.order == 2) q2_tables(c.q2, m.h);
}

size_t elem_lin_doubles(const ElemCtx& c) {
  const int dim = c.m.dim;
  if (dim == 3 && c.m.order == 2)  // [tile][coefficient][element warp][32 lanes: 27 Gauss points]
    return (size_t)c.ntx * c.nty * c.ntz * (Q2HexTile::X * Q2HexTile::Y * Q2HexTile::Z) * 32 * c.nlin;
  const size_t ne_tile = dim == 3 ? Tile<3>::X * Tile<3>::Y * Tile<3>::Z : Tile<2>::X * Tile<2>::Y;
  const size_t ng = c.m.order == 2 ? 9 : (dim == 3 ? 8 : 4);
  return (size_t)c.ntx * c.nty * c.ntz * ne_tile * ng * c.nlin;
}

template <int DIM, int MODEL, int MODE>
static cudaError_t run_colours(const ElemCtx& c, ElemArgs a, cudaStream_t st) {
  constexpr int NE = Tile<DIM>::X * Tile<DIM>::Y * Tile<DIM>::Z;
  // 3D: tile-level sum factorisation for the tangent and residual passes
  constexpr bool tan3 = DIM == 3 && (MODE == M_JV || MODE == M_JTV);
  constexpr bool res3 = DIM == 3 && (MODE == M_RES || MODE == M_RES_LIN);
  // the residual stages phi^n with gradients and phihat_old only where the time term or the
  // Eq. (theta) estimate uses them (Res3L<true>); otherwise the smaller layout
  const bool ext = a.P.time_form != 0 || (a.P.phihat_old && a.phold);
  if constexpr (res3) {
    const cudaError_t e =
        ext ? cudaFuncSetAttribute(res3_kernel<MODEL, MODE == M_RES_LIN, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Res3L<true>::BYTES)
            : cudaFuncSetAttribute(res3_kernel<MODEL, MODE == M_RES_LIN, false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Res3L<false>::BYTES);
    if (e != cudaSuccess) return e;
  }
  for (int col = 0; col < (1 << DIM); ++col) {
    const int cx = col & 1, cy = (col >> 1) & 1, cz = (col >> 2) & 1;
    a.color = col;
    a.ctx = (c.ntx - cx + 1) / 2;
    a.cty = (c.nty - cy + 1) / 2;
    a.ctz = DIM == 3 ? (c.ntz - cz + 1) / 2 : 1;
    const long long blocks = (long long)a.ctx * a.cty * a.ctz;
    if (blocks <= 0) continue;
    cudaError_t e;
    if constexpr (tan3)
      e = launch_colour(tan3_kernel<MODEL, MODE == M_JTV>, (unsigned)blocks, T3::NE, Tan3::BYTES, st, col > 0, a);
    else if constexpr (res3)
      e = ext ? launch_colour(res3_kernel<MODEL, MODE == M_RES_LIN, true>, (unsigned)blocks, T3::NE,
                              Res3L<true>::BYTES, st, col > 0, a)
              : launch_colour(res3_kernel<MODEL, MODE == M_RES_LIN, false>, (unsigned)blocks, T3::NE,
                              Res3L<false>::BYTES, st, col > 0, a);
    else
      e = launch_colour(elem_kernel<DIM, MODEL, MODE>, (unsigned)blocks, NE, 0, st, col > 0, a);
    if (e != cudaSuccess) return e;
    count_launches(1);
  }
  return cudaGetLastError();
}

template <int DIM, int MODEL>
static cudaError_t dispatch_mode(int mode, const ElemCtx& c, const ElemArgs& a, cudaStream_t st) {
  switch (mode) {
    case M_RES: return run_colours<DIM, MODEL, M_RES>(c, a, st);
    case M_RES_LIN: return run_colours<DIM, MODEL, M_RES_LIN>(c, a, st);
    case M_JV: return run_colours<DIM, MODEL, M_JV>(c, a, st);
    case M_JTV: return run_colours<DIM, MODEL, M_JTV>(c, a, st);
    case M_DEPS: return run_colours<DIM, MODEL, M_DEPS>(c, a, st);
    case M_PREV_T: return run_colours<DIM, MODEL, M_PREV_T>(c, a, st);
    case M_OLD: return run_colours<DIM, MODEL, M_OLD>(c, a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t elem_run(int mode, const ElemCtx& c, const double* U, const double* Un, const double* V, double* out,
                     double* lin, cudaStream_t st, const double* init, const double* phold) {
  cudaError_t e = init ? cudaMemcpyAsync(out, init, sizeof(double) * 2 * (size_t)c.m.nn, cudaMemcpyDeviceToDevice, st)
                       : cudaMemsetAsync(out, 0, sizeof(double) * 2 * (size_t)c.m.nn, st);
  if (e != cudaSuccess) return e;
  if (c.m.order == 2 && c.m.dim == 3) return q2h_run(mode, c, U, Un, V, out, lin, st, phold);
  if (c.m.order == 2) return q2_run(mode, c, U, Un, V, out, lin, st, phold);
  ElemArgs a;
  a.m = c.m;
  a.P = c.P;
  a.h = c.m.h;
  a.inv_h = 1.0 / c.m.h;
  a.wh = (c.m.dim == 3 ? 0.125 * c.m.h * c.m.h : 0.25 * c.m.h);
  a.K = c.K;
  a.C = c.m.dim == 3 ? c.pw_res3 : c.pw_elem;
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
  if (c.m.dim == 3) {
    return c.P.model == 0 ? dispatch_mode<3, 0>(mode, c, a, st) : dispatch_mode<3, 1>(mode, c, a, st);
  }
  return c.P.model == 0 ? dispatch_mode<2, 0>(mode, c, a, st) : dispatch_mode<2, 1>(mode, c, a, st);
}

}  // namespace tusas
