// 3D element passes with tile-level sum factorisation (tangent, transposed
// tangent, residual, residual + linearisation).
//
// The staged 1D forms of interp_l / accumulate_l work axis by axis, and the
// x- and y-stages of an element only see the nodes of one x-edge or one face:
// neighbouring elements of a tile share them. These kernels run those stages
// once per edge / face of the 8 x 4 x 4 tile through shared memory instead of
// once per element: forward, x-stage per x-edge, y-stage per xy-face, z-stage
// per element; after the pointwise integrands the transposed z-stage per
// element, contributions summed per face, transposed y-stage per face, summed
// per x-edge, transposed x-stage per x-edge, summed per node. The operations
// on every quantity are those of interp_l (bitwise the same Gauss-point
// values) and of accumulate_l up to the order of the sums. Per element and
// field this takes about 40 FP64 operations for values and gradients (54 per
// element alone), 24 for values alone (36), and about 76 for the accumulation
// with the node sums (90).
//
// Included by residual.cu inside namespace tusas, after ElemArgs.
#pragma once

struct T3 {
  static const int TX = Tile<3>::X, TY = Tile<3>::Y, TZ = Tile<3>::Z;
  static const int NX = TX + 1, NY = TY + 1, NZ = TZ + 1;
  static const int NT = NX * NY * NZ;  // nodes
  static const int NE = TX * TY * TZ;  // elements = threads
  static const int UX = TX * NY * NZ;  // x-edges (ex, ny, nz)
  static const int UY = TX * TY * NZ;  // xy-faces (ex, ey, nz)
  // transposed buffers (doubles), aliased over the forward ones once those are read
  static const int ZC = 32 * NE;  // [2 fields][2 levels][8][NE]
  static const int YC = 12 * UY;  // [2 fields][2 slots][3][UY]
  static const int XC = 4 * UX;   // [2 fields][2 slots][UX]
  static const int BWD = ZC + YC;
  // forward buffers of one field: x-stage (3 or 2 arrays of UX), y-stage (8 or 4 of UY)
  static const int XG = 3 * UX, XV = 2 * UX, YG = 8 * UY, YV = 4 * UY;
};

// ---- forward stages, one field ----------------------------------------------------
// x-stage per x-edge: [0] value at the lower x Gauss point, [1] upper, [2] difference (GRAD)
template <bool GRAD>
__device__ __forceinline__ void t3_x(const double* sN, double* X, int tid) {
  const double t = TUSAS_GP_T;
  for (int u = tid; u < T3::UX; u += T3::NE) {
    const int n0 = u % T3::TX + T3::NX * (u / T3::TX);
    const double x0 = sN[n0], x1 = sN[n0 + 1];
    const double bb = x1 - x0;
    X[u] = fma(t, bb, x0);
    X[T3::UX + u] = fma(-t, bb, x1);
    if (GRAD) X[2 * T3::UX + u] = bb;
  }
}

// y-stage per xy-face from the x-edges at ny = ey, ey + 1: [0..3] values at
// (x bit, y bit) = (k & 1, k >> 1); GRAD: [4, 5] y-differences at x bit, [6, 7] x-differences at y bit
template <bool GRAD>
__device__ __forceinline__ void t3_y(const double* X, double* Y, int tid) {
  constexpr int TX = T3::TX, TY = T3::TY, NY = T3::NY, UX = T3::UX, UY = T3::UY;
  const double t = TUSAS_GP_T;
  for (int u = tid; u < UY; u += T3::NE) {
    const int ex = u % TX, ey = (u / TX) % TY, nz = u / (TX * TY);
    const int lo = ex + TX * (ey + NY * nz), hi = lo + TX;
    if (GRAD) {  // x-differences along y first (the order of interp_l)
      const double x0 = X[2 * UX + lo], x1 = X[2 * UX + hi];
      const double bb = x1 - x0;
      Y[6 * UY + u] = fma(t, bb, x0);
      Y[7 * UY + u] = fma(-t, bb, x1);
    }
#pragma unroll
    for (int xb = 0; xb < 2; ++xb) {
      const double x0 = X[xb * UX + lo], x1 = X[xb * UX + hi];
      const double bb = x1 - x0;
      if (GRAD) Y[(4 + xb) * UY + u] = bb;
      Y[xb * UY + u] = fma(t, bb, x0);
      Y[(xb + 2) * UY + u] = fma(-t, bb, x1);
    }
  }
}

// z-stage of element tid from the faces below and above it: val[g] and, if GRAD,
// grd[d][j] = h dv/dx_d at the Gauss points whose other-axis bits are j (interp_l's layout)
template <bool GRAD>
__device__ __forceinline__ void t3_z(const double* Y, int tid, double* val, double (*grd)[4]) {
  constexpr int UY = T3::UY;
  const double t = TUSAS_GP_T;
  const int u0 = tid, u1 = tid + T3::TX * T3::TY;
  if (GRAD) {
#pragma unroll
    for (int yb = 0; yb < 2; ++yb) {  // x-differences along z: grd[0][y + 2 z]
      const double x0 = Y[(6 + yb) * UY + u0], x1 = Y[(6 + yb) * UY + u1];
      const double bb = x1 - x0;
      grd[0][yb] = fma(t, bb, x0);
      grd[0][yb + 2] = fma(-t, bb, x1);
    }
#pragma unroll
    for (int xb = 0; xb < 2; ++xb) {  // y-differences along z: grd[1][x + 2 z]
      const double x0 = Y[(4 + xb) * UY + u0], x1 = Y[(4 + xb) * UY + u1];
      const double bb = x1 - x0;
      grd[1][xb] = fma(t, bb, x0);
      grd[1][xb + 2] = fma(-t, bb, x1);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {  // values along z; z-differences grd[2][x + 2 y]
    const double x0 = Y[k * UY + u0], x1 = Y[k * UY + u1];
    const double bb = x1 - x0;
    if (GRAD) grd[2][k] = bb;
    val[k] = fma(t, bb, x0);
    val[k + 4] = fma(-t, bb, x1);
  }
}

// The z-stage split by Gauss-point column, the same operations as t3_z: gx[y + 2 z] and
// gy[x + 2 z] are the x- and y-differences interpolated along z (grd[0], grd[1] of t3_z) ...
__device__ __forceinline__ void t3_zxy(const double* Y, int tid, double* gx, double* gy) {
  constexpr int UY = T3::UY;
  const double t = TUSAS_GP_T;
  const int u0 = tid, u1 = tid + T3::TX * T3::TY;
#pragma unroll
  for (int yb = 0; yb < 2; ++yb) {
    const double x0 = Y[(6 + yb) * UY + u0], x1 = Y[(6 + yb) * UY + u1];
    const double bb = x1 - x0;
    gx[yb] = fma(t, bb, x0);
    gx[yb + 2] = fma(-t, bb, x1);
  }
#pragma unroll
  for (int xb = 0; xb < 2; ++xb) {
    const double x0 = Y[(4 + xb) * UY + u0], x1 = Y[(4 + xb) * UY + u1];
    const double bb = x1 - x0;
    gy[xb] = fma(t, bb, x0);
    gy[xb + 2] = fma(-t, bb, x1);
  }
}
// ... and v0, v1 the values at the Gauss points (k, z = 0) and (k, z = 1) of column
// k = x + 2 y, dz their z-difference (val[k], val[k + 4], grd[2][k] of t3_z).
__device__ __forceinline__ void t3_zcol(const double* Y, int tid, int k, double& v0, double& v1, double& dz) {
  constexpr int UY = T3::UY;
  const double t = TUSAS_GP_T;
  const double x0 = Y[k * UY + tid], x1 = Y[k * UY + tid + T3::TX * T3::TY];
  const double bb = x1 - x0;
  dz = bb;
  v0 = fma(t, bb, x0);
  v1 = fma(-t, bb, x1);
}

// ---- transposed stages ----------------------------------------------------------------
// Transposed z-stage of one element and field from the integrands sv at the Gauss points and
// the flux pair sums F[d][j] = f_d at the two Gauss points along d (accumulated while the
// Gauss points are evaluated, which keeps 12 instead of 24 flux values live per field):
// contributions to the face below (lo) and above (hi) in the face layout.
__device__ __forceinline__ void t3_zt_sums(const double* sv, double (*F)[4], double* lo, double* hi) {
  const double t = TUSAS_GP_T;
#pragma unroll
  for (int k = 0; k < 4; ++k) {  // values with the z-differences
    const double yL = sv[k], yR = sv[k + 4];
    const double q = fma(t, yL - yR, F[2][k]);
    lo[k] = yL - q;
    hi[k] = yR + q;
  }
#pragma unroll
  for (int yb = 0; yb < 2; ++yb) {  // x-differences: transposed interpolation along z
    const double yL = F[0][yb], yR = F[0][yb + 2];
    const double dd = yL - yR;
    lo[6 + yb] = fma(-t, dd, yL);
    hi[6 + yb] = fma(t, dd, yR);
  }
#pragma unroll
  for (int xb = 0; xb < 2; ++xb) {  // y-differences
    const double yL = F[1][xb], yR = F[1][xb + 2];
    const double dd = yL - yR;
    lo[4 + xb] = fma(-t, dd, yL);
    hi[4 + xb] = fma(t, dd, yR);
  }
}

// flux of Gauss point g into the pair sums: F[d][j] = f_d(g with bit d clear) + f_d(g with bit d set)
__device__ __forceinline__ void t3_flux_sum(double (*F)[4], const double* f, int g) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if ((g >> d) & 1)
      F[d][remove_bit(g, d)] += f[d];
    else
      F[d][remove_bit(g, d)] = f[d];
  }
}

// Tile-level transposed y- and x-stages and node sums of the two output fields, given
// each element's transposed z-stage outputs (zlo, zhi; zero for elements outside the
// mesh). Starts with a barrier: the shared buffers alias the forward ones. The node
// sums are multiplied by `scale` if SCALE and added to out.
template <bool SCALE>
__device__ __forceinline__ void t3_tile_t(double* sm, const double (*zlo)[8], const double (*zhi)[8], int tid,
                                          const DevMesh& m, int ex0, int ey0, int ez0, double scale, double* out) {
  constexpr int TX = T3::TX, TY = T3::TY, TZ = T3::TZ, NX = T3::NX, NY = T3::NY;
  constexpr int NT = T3::NT, NE = T3::NE, UX = T3::UX, UY = T3::UY;
  const double t = TUSAS_GP_T;
  double* sZc = sm;
  double* sYc = sm + T3::ZC;
  double* sXc = sm;
  __syncthreads();  // every forward read is done
#pragma unroll
  for (int f = 0; f < 2; ++f) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      sZc[((f * 2 + 0) * 8 + k) * NE + tid] = zlo[f][k];
      sZc[((f * 2 + 1) * 8 + k) * NE + tid] = zhi[f][k];
    }
  }
  __syncthreads();

  // per face: the element above (its lower level) plus the element below (upper level),
  // transposed y-stage to the x-edges at ny = ey (slot 0) and ey + 1 (slot 1)
  for (int u = tid; u < UY; u += NE) {
    const int nz = u / (TX * TY);  // uniform across a warp (32 faces per level)
    const int e_up = u, e_dn = u - TX * TY;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      double c[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double a = nz < TZ ? sZc[((f * 2 + 0) * 8 + k) * NE + e_up] : 0.0;
        c[k] = nz > 0 ? a + sZc[((f * 2 + 1) * 8 + k) * NE + e_dn] : a;
      }
      double* Yc = sYc + 6 * f * UY;  // [slot][X0, X1, Xb][u]
#pragma unroll
      for (int xb = 0; xb < 2; ++xb) {
        const double yL = c[xb], yR = c[xb + 2];
        const double q = fma(t, yL - yR, c[4 + xb]);
        Yc[(0 * 3 + xb) * UY + u] = yL - q;
        Yc[(1 * 3 + xb) * UY + u] = yR + q;
      }
      const double dd = c[6] - c[7];
      Yc[(0 * 3 + 2) * UY + u] = fma(-t, dd, c[6]);
      Yc[(1 * 3 + 2) * UY + u] = fma(t, dd, c[7]);
    }
  }
  __syncthreads();

  // per x-edge (ex, ny, nz): the faces on both sides in y, transposed x-stage
  for (int u = tid; u < UX; u += NE) {
    const int ex = u % TX, ny = (u / TX) % NY, nz = u / (TX * NY);
    const int fa = ex + TX * (ny + TY * nz);  // face (ex, ny, nz): slot 0
    const int fb = fa - TX;                   // face (ex, ny - 1, nz): slot 1
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double* Yc = sYc + 6 * f * UY;
      double c[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double a = ny < TY ? Yc[(0 * 3 + k) * UY + fa] : 0.0;
        const double bb = ny > 0 ? Yc[(1 * 3 + k) * UY + fb] : 0.0;
        c[k] = a + bb;
      }
      const double q = fma(t, c[0] - c[1], c[2]);
      sXc[(f * 2 + 0) * UX + u] = c[0] - q;
      sXc[(f * 2 + 1) * UX + u] = c[1] + q;
    }
  }
  __syncthreads();

  // node sums in fixed order, read-modify-write. The previous tile colour writes the same
  // boundary nodes: a colour launched as a programmatic dependent of the previous one waits
  // here, and only here, for that grid to complete and its writes to be visible (a no-op
  // after an ordinary launch); the reads bypass L1, which may hold lines of an earlier colour.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int s = tid; s < NT; s += NE) {
    const int nx_ = s % NX, r = s / NX;
    const int ny_ = r % NY, nz_ = r / NY;
    const int gx = ex0 + nx_, gy = ey0 + ny_, gz = ez0 + nz_;
    if (gx >= m.nnx || gy >= m.nny || gz >= m.nnz) continue;
    const int ea = nx_ + TX * r;  // edge (nx, ny, nz): left node, slot 0
    const int eb = ea - 1;        // edge (nx - 1, ny, nz): right node, slot 1
    double acc[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double a = nx_ < TX ? sXc[(f * 2 + 0) * UX + ea] : 0.0;
      const double bb = nx_ > 0 ? sXc[(f * 2 + 1) * UX + eb] : 0.0;
      acc[f] = a + bb;
      if (SCALE) acc[f] *= scale;
    }
    const i64 node = gx + (i64)m.nnx * (gy + (i64)m.nny * gz);
    out[node] = __ldcg(out + node) + acc[0];
    out[m.nn + node] = __ldcg(out + m.nn + node) + acc[1];
  }
}

// tile coordinates of this block (colour-strided tile grid)
struct T3Tile {
  int tx, ty, tz, ex0, ey0, ez0;
  __device__ __forceinline__ T3Tile(const ElemArgs& A) {
    int b = blockIdx.x;
    const int ix = b % A.ctx;
    b /= A.ctx;
    const int iy = b % A.cty;
    const int iz = b / A.cty;
    tx = 2 * ix + (A.color & 1);
    ty = 2 * iy + ((A.color >> 1) & 1);
    tz = 2 * iz + ((A.color >> 2) & 1);
    ex0 = tx * T3::TX;
    ey0 = ty * T3::TY;
    ez0 = tz * T3::TZ;
  }
};

// stage one nodal field of the tile (zero outside the mesh); x = f(node) for in-mesh nodes
template <typename F>
__device__ __forceinline__ void t3_stage(double* sN, const DevMesh& m, const T3Tile& T, int tid, F x) {
  for (int s = tid; s < T3::NT; s += T3::NE) {
    const int lx = s % T3::NX, ly = (s / T3::NX) % T3::NY, lz = s / (T3::NX * T3::NY);
    const int gx = T.ex0 + lx, gy = T.ey0 + ly, gz = T.ez0 + lz;
    const bool ok = gx < m.nnx && gy < m.nny && gz < m.nnz;
    sN[s] = ok ? x(gx + (i64)m.nnx * (gy + (i64)m.nny * gz)) : 0.0;
  }
}

// ---- tangent J v (TRANS = false) and J^T w (TRANS = true) ------------------------------
struct Tan3 {
  static const int OFF_X = 2 * T3::NT;             // [2][3][UX], after the staged nodes
  static const int OFF_Y = OFF_X + 2 * T3::XG;     // [2][8][UY]
  static const int FWD = OFF_Y + 2 * T3::YG;
  static const int DOUBLES = FWD > T3::BWD ? FWD : T3::BWD;
  static const size_t BYTES = sizeof(double) * DOUBLES;
};
static_assert(Tan3::BYTES <= 48 * 1024, "tan3_kernel launches without the large-shared-memory opt-in");

// 4 CTAs per SM (128 registers): with the flux pair sums accumulated per Gauss point the
// tangent fits with at most 56 bytes of spills (8.05 -> 8.01 ms per application on the alloy
// box against 3 CTAs; 2 CTAs per SM cost 13 %)
template <int MODEL, bool TRANS>
__global__ void __launch_bounds__(T3::NE, 4) tan3_kernel(const ElemArgs A) {
  constexpr int NE = T3::NE;
  constexpr int NC = NLin<3, MODEL>::VALUE;
  extern __shared__ double sm[];
  const DevMesh& m = A.m;
  const T3Tile T(A);
  const int tid = threadIdx.x;
  double* sN = sm;
  double* sX = sm + Tan3::OFF_X;
  double* sY = sm + Tan3::OFF_Y;
  // the next tile colour may start on free SMs now: it touches nothing this grid writes
  // before its own wait at the node sums
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  t3_stage(sN, m, T, tid, [&](i64 n) { return A.V[n]; });
  t3_stage(sN + T3::NT, m, T, tid, [&](i64 n) { return A.V[m.nn + n]; });
  __syncthreads();
  t3_x<true>(sN, sX, tid);
  t3_x<true>(sN + T3::NT, sX + T3::XG, tid);
  __syncthreads();
  t3_y<true>(sX, sY, tid);
  t3_y<true>(sX + T3::XG, sY + T3::YG, tid);
  __syncthreads();

  const int lx = tid % T3::TX, ly = (tid / T3::TX) % T3::TY, lz = tid / (T3::TX * T3::TY);
  const bool valid = T.ex0 + lx < m.nx && T.ey0 + ly < m.ny && T.ez0 + lz < m.nz;
  double zlo[2][8], zhi[2][8];
  if (valid) {
    // Gauss points by column k = x + 2 y, as in res3_kernel (same operations and order)
    double g0x[4], g0y[4], g1x[4], g1y[4];
    t3_zxy(sY, tid, g0x, g0y);
    t3_zxy(sY + T3::YG, tid, g1x, g1y);
    const i64 tile_id = T.tx + (i64)A.ntx * (T.ty + (i64)A.nty * T.tz);
    const double* linp = A.lin + tile_id * (i64)(NC * 8 * NE) + tid;  // [c][g][t] within the tile
    double Fx0[4], Fy0[4], Fx1[4], Fy1[4];
    GPOut<3> o;
    const double t = TUSAS_GP_T;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int x = k & 1, y = k >> 1;
      double v0[2], v1[2], z0, z1;
      t3_zcol(sY, tid, k, v0[0], v0[1], z0);
      t3_zcol(sY + T3::YG, tid, k, v1[0], v1[1], z1);
      double sv0[2], sv1[2], fz0[2], fz1[2];
#pragma unroll
      for (int zb = 0; zb < 2; ++zb) {
        const int g = k + 4 * zb;
        double L[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) L[c] = __ldg(linp + (c * 8 + g) * NE);
        const double xp[3] = {g0x[y + 2 * zb], g0y[x + 2 * zb], z0};
        const double xg[3] = {g1x[y + 2 * zb], g1y[x + 2 * zb], z1};
        lin_apply<3, MODEL, TRANS, true>(A.P, L, v0[zb], v1[zb], xp, xg, o, A.K);
        sv0[zb] = o.sphi;
        sv1[zb] = o.su;
        fz0[zb] = o.fphi[2];
        fz1[zb] = o.fu[2];
        if (x == 0) {
          Fx0[y + 2 * zb] = o.fphi[0];
          Fx1[y + 2 * zb] = o.fu[0];
        } else {
          Fx0[y + 2 * zb] += o.fphi[0];
          Fx1[y + 2 * zb] += o.fu[0];
        }
        if (y == 0) {
          Fy0[x + 2 * zb] = o.fphi[1];
          Fy1[x + 2 * zb] = o.fu[1];
        } else {
          Fy0[x + 2 * zb] += o.fphi[1];
          Fy1[x + 2 * zb] += o.fu[1];
        }
      }
      double F2 = fz0[0];
      F2 += fz0[1];
      double q = fma(t, sv0[0] - sv0[1], F2);
      zlo[0][k] = sv0[0] - q;
      zhi[0][k] = sv0[1] + q;
      F2 = fz1[0];
      F2 += fz1[1];
      q = fma(t, sv1[0] - sv1[1], F2);
      zlo[1][k] = sv1[0] - q;
      zhi[1][k] = sv1[1] + q;
    }
#pragma unroll
    for (int yb = 0; yb < 2; ++yb) {
      double dd = Fx0[yb] - Fx0[yb + 2];
      zlo[0][6 + yb] = fma(-t, dd, Fx0[yb]);
      zhi[0][6 + yb] = fma(t, dd, Fx0[yb + 2]);
      dd = Fx1[yb] - Fx1[yb + 2];
      zlo[1][6 + yb] = fma(-t, dd, Fx1[yb]);
      zhi[1][6 + yb] = fma(t, dd, Fx1[yb + 2]);
    }
#pragma unroll
    for (int xb = 0; xb < 2; ++xb) {
      double dd = Fy0[xb] - Fy0[xb + 2];
      zlo[0][4 + xb] = fma(-t, dd, Fy0[xb]);
      zhi[0][4 + xb] = fma(t, dd, Fy0[xb + 2]);
      dd = Fy1[xb] - Fy1[xb + 2];
      zlo[1][4 + xb] = fma(-t, dd, Fy1[xb]);
      zhi[1][4 + xb] = fma(t, dd, Fy1[xb + 2]);
    }
  } else {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
#pragma unroll
      for (int k = 0; k < 8; ++k) zlo[f][k] = zhi[f][k] = 0.0;
    }
  }
  t3_tile_t<false>(sm, zlo, zhi, tid, m, T.ex0, T.ey0, T.ez0, 1.0, A.out);
}

// ---- residual (LIN = false) and residual + stored linearisation (LIN = true) -----------
// Nodal fields: phi, u (with gradients), phi - phi^n, u - u^n (values), and with EXT phi^n
// (with gradients, for the difference-of-products time term) and phihat_old (values, for the
// Eq. (theta) estimate), staged only when used. Without EXT the layout holds the first four:
// 48 KB instead of 70 KB per CTA.
template <bool EXT>
struct Res3L {
  static const int NF = EXT ? 6 : 4;
  static const int OFF_X = 0;                                   // x-stage of the NF fields
  static const int X_PHI = 0, X_U = T3::XG, X_DP = 2 * T3::XG, X_DU = X_DP + T3::XV, X_PN = X_DU + T3::XV,
                   X_PO = X_PN + T3::XG;
  static const int XS = EXT ? X_PO + T3::XV : X_PN;
  static const int OFF_N = XS;                                  // staged nodes [NF][NT]
  static const int OFF_Y = XS;                                  // y-stage (aliases the nodes)
  static const int Y_PHI = 0, Y_U = T3::YG, Y_DP = 2 * T3::YG, Y_DU = Y_DP + T3::YV, Y_PN = Y_DU + T3::YV,
                   Y_PO = Y_PN + T3::YG;
  static const int YS = EXT ? Y_PO + T3::YV : Y_PN;
  static const int NS = NF * T3::NT;
  static const int FWD = XS + (YS > NS ? YS : NS);
  static const int DOUBLES = FWD > T3::BWD ? FWD : T3::BWD;
  static const size_t BYTES = sizeof(double) * DOUBLES;
};

// The residual runs 3 CTAs per SM with the EXT layout and 4 without: with the Gauss points
// taken by column it needs 152 registers (all eight points' interpolated inputs at once
// needed 206, and forcing 3 CTAs then spilled); the linearisation pass, 200 registers, runs 2.
template <int MODEL, bool LIN, bool EXT>
__global__ void __launch_bounds__(T3::NE, (LIN ? 2 : (EXT ? 3 : 4))) res3_kernel(const ElemArgs A) {
  constexpr int NE = T3::NE, NT = T3::NT;
  constexpr int NC = NLin<3, MODEL>::VALUE;
  using Res3 = Res3L<EXT>;
  extern __shared__ double sm[];
  const DevMesh& m = A.m;
  const T3Tile T(A);
  const int tid = threadIdx.x;
  const bool tf1 = EXT && A.P.time_form != 0;
  const bool pho_on = EXT && A.P.phihat_old && A.phold;
  // the next tile colour may start on free SMs now (it waits at the node sums)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  double* sN = sm + Res3::OFF_N;
  double* sX = sm + Res3::OFF_X;
  double* sY = sm + Res3::OFF_Y;

  t3_stage(sN, m, T, tid, [&](i64 n) { return A.U[n]; });
  t3_stage(sN + NT, m, T, tid, [&](i64 n) { return A.U[m.nn + n]; });
  t3_stage(sN + 2 * NT, m, T, tid, [&](i64 n) { return A.U[n] - A.Un[n]; });
  t3_stage(sN + 3 * NT, m, T, tid, [&](i64 n) { return A.U[m.nn + n] - A.Un[m.nn + n]; });
  if (tf1) t3_stage(sN + 4 * NT, m, T, tid, [&](i64 n) { return A.Un[n]; });
  if (pho_on) t3_stage(sN + 5 * NT, m, T, tid, [&](i64 n) { return A.phold[n]; });
  __syncthreads();
  t3_x<true>(sN, sX + Res3::X_PHI, tid);
  t3_x<true>(sN + NT, sX + Res3::X_U, tid);
  t3_x<false>(sN + 2 * NT, sX + Res3::X_DP, tid);
  t3_x<false>(sN + 3 * NT, sX + Res3::X_DU, tid);
  if (tf1) t3_x<true>(sN + 4 * NT, sX + Res3::X_PN, tid);
  if (pho_on) t3_x<false>(sN + 5 * NT, sX + Res3::X_PO, tid);
  __syncthreads();  // the y-stage overwrites the staged nodes
  t3_y<true>(sX + Res3::X_PHI, sY + Res3::Y_PHI, tid);
  t3_y<true>(sX + Res3::X_U, sY + Res3::Y_U, tid);
  t3_y<false>(sX + Res3::X_DP, sY + Res3::Y_DP, tid);
  t3_y<false>(sX + Res3::X_DU, sY + Res3::Y_DU, tid);
  if (tf1) t3_y<true>(sX + Res3::X_PN, sY + Res3::Y_PN, tid);
  if (pho_on) t3_y<false>(sX + Res3::X_PO, sY + Res3::Y_PO, tid);
  __syncthreads();

  const int lx = tid % T3::TX, ly = (tid / T3::TX) % T3::TY, lz = tid / (T3::TX * T3::TY);
  const int ez = T.ez0 + lz;
  const bool valid = T.ex0 + lx < m.nx && T.ey0 + ly < m.ny && ez < m.nz;
  double zlo[2][8], zhi[2][8];
  if (valid) {
    // Gauss points by column k = x + 2 y, the pair (k, z = 0), (k, z = 1) at a time: the values
    // and z-differences of a column come from the faces when it is reached and its
    // transposed z-stage follows its integrands, so only the x- and y-differences and the
    // flux pair sums live across the loop. Operations and summation order are those of
    // t3_z, t3_flux_sum and t3_zt_sums over the Gauss points in order.
    double gpx[4], gpy[4], gux[4], guy[4], gnx[4] = {0, 0, 0, 0}, gny[4] = {0, 0, 0, 0};
    t3_zxy(sY + Res3::Y_PHI, tid, gpx, gpy);
    t3_zxy(sY + Res3::Y_U, tid, gux, guy);
    if (tf1) t3_zxy(sY + Res3::Y_PN, tid, gnx, gny);
    const i64 tile_id = T.tx + (i64)A.ntx * (T.ty + (i64)A.nty * T.tz);
    double* linp = A.lin + tile_id * (i64)(NC * 8 * NE) + tid;  // [c][g][t] within the tile
    // flux pair sums: x-fluxes summed over x at (y, z), y-fluxes over y at (x, z)
    double Fx0[4], Fy0[4], Fx1[4], Fy1[4];
    GPOut<3> o;
    // frozen gradient at the two Gauss-point levels of the element (z = z0 + h (ez + t), h (ez + 1 - t))
    double G4z[2] = {0.0, 0.0};
    if (MODEL == 1 && A.P.has_g4) {
      G4z[0] = fma(fma(m.h, ez + TUSAS_GP_T, m.z0), A.C.ilT, A.C.g4off);
      G4z[1] = fma(fma(m.h, ez + (1.0 - TUSAS_GP_T), m.z0), A.C.ilT, A.C.g4off);
    }
    const double t = TUSAS_GP_T;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int x = k & 1, y = k >> 1;
      double ph[2], uu[2], dph[2], duu[2], po[2] = {0.0, 0.0}, pz, uz, pnz = 0.0, dummy;
      t3_zcol(sY + Res3::Y_PHI, tid, k, ph[0], ph[1], pz);
      t3_zcol(sY + Res3::Y_U, tid, k, uu[0], uu[1], uz);
      t3_zcol(sY + Res3::Y_DP, tid, k, dph[0], dph[1], dummy);
      t3_zcol(sY + Res3::Y_DU, tid, k, duu[0], duu[1], dummy);
      if (tf1) {
        double a0, a1;
        t3_zcol(sY + Res3::Y_PN, tid, k, a0, a1, pnz);
      }
      if (pho_on) t3_zcol(sY + Res3::Y_PO, tid, k, po[0], po[1], dummy);
      double sv0[2], sv1[2], fz0[2], fz1[2];
#pragma unroll
      for (int zb = 0; zb < 2; ++zb) {
        const int g = k + 4 * zb;
        // gradients stay in the staged units (h times the gradient): A.C carries the factors
        const double p[3] = {gpx[y + 2 * zb], gpy[x + 2 * zb], pz};
        const double gg[3] = {gux[y + 2 * zb], guy[x + 2 * zb], uz};
        const double pn[3] = {gnx[y + 2 * zb], gny[x + 2 * zb], pnz};
        double L[LIN ? NC : 1];
        pointwise<3, MODEL, LIN>(A.P, A.C, ph[zb], uu[zb], dph[zb], duu[zb], po[zb], p, gg, pn, G4z[zb], o, L, A.K);
        if (LIN) {
#pragma unroll
          for (int c = 0; c < NC; ++c) linp[(c * 8 + g) * NE] = L[c];
        }
        // true-unit integrands: values times h here, the node sums times w / h
        sv0[zb] = o.sphi * A.h;
        sv1[zb] = o.su * A.h;
        fz0[zb] = o.fphi[2];
        fz1[zb] = o.fu[2];
        if (x == 0) {
          Fx0[y + 2 * zb] = o.fphi[0];
          Fx1[y + 2 * zb] = o.fu[0];
        } else {
          Fx0[y + 2 * zb] += o.fphi[0];
          Fx1[y + 2 * zb] += o.fu[0];
        }
        if (y == 0) {
          Fy0[x + 2 * zb] = o.fphi[1];
          Fy1[x + 2 * zb] = o.fu[1];
        } else {
          Fy0[x + 2 * zb] += o.fphi[1];
          Fy1[x + 2 * zb] += o.fu[1];
        }
      }
      // transposed z-stage of the values of column k (the z-flux pair sum as in t3_flux_sum)
      double F2 = fz0[0];
      F2 += fz0[1];
      double q = fma(t, sv0[0] - sv0[1], F2);
      zlo[0][k] = sv0[0] - q;
      zhi[0][k] = sv0[1] + q;
      F2 = fz1[0];
      F2 += fz1[1];
      q = fma(t, sv1[0] - sv1[1], F2);
      zlo[1][k] = sv1[0] - q;
      zhi[1][k] = sv1[1] + q;
    }
    // x- and y-differences transposed along z (the tail of t3_zt_sums)
#pragma unroll
    for (int yb = 0; yb < 2; ++yb) {
      double dd = Fx0[yb] - Fx0[yb + 2];
      zlo[0][6 + yb] = fma(-t, dd, Fx0[yb]);
      zhi[0][6 + yb] = fma(t, dd, Fx0[yb + 2]);
      dd = Fx1[yb] - Fx1[yb + 2];
      zlo[1][6 + yb] = fma(-t, dd, Fx1[yb]);
      zhi[1][6 + yb] = fma(t, dd, Fx1[yb + 2]);
    }
#pragma unroll
    for (int xb = 0; xb < 2; ++xb) {
      double dd = Fy0[xb] - Fy0[xb + 2];
      zlo[0][4 + xb] = fma(-t, dd, Fy0[xb]);
      zhi[0][4 + xb] = fma(t, dd, Fy0[xb + 2]);
      dd = Fy1[xb] - Fy1[xb + 2];
      zlo[1][4 + xb] = fma(-t, dd, Fy1[xb]);
      zhi[1][4 + xb] = fma(t, dd, Fy1[xb + 2]);
    }
  } else {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
#pragma unroll
      for (int k = 0; k < 8; ++k) zlo[f][k] = zhi[f][k] = 0.0;
    }
  }
  t3_tile_t<true>(sm, zlo, zhi, tid, m, T.ex0, T.ey0, T.ez0, A.wh, A.out);
}
