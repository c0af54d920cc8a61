// 3D tangent and transposed-tangent passes with tile-level sum factorisation.
//
// The staged 1D forms of interp_l / accumulate_l work axis by axis, and the
// x- and y-stages of an element only see the nodes of one x-edge or one face:
// neighbouring elements of a tile share them. This kernel runs those stages
// once per edge / face of the tile through shared memory instead of once per
// element: forward, x-stage per x-edge (3 values), y-stage per xy-face (8),
// z-stage per element; after the pointwise product the transposed z-stage per
// element, contributions summed per face, transposed y-stage per face, summed
// per x-edge, transposed x-stage per x-edge, summed per node. The operations
// on every quantity are those of interp_l (bitwise the same Gauss-point
// values) and of accumulate_l up to the order of the sums. Per element and
// field this takes about 40 FP64 operations for the interpolation (54 per
// element alone) and about 74 for the accumulation with the node sums (90).
// Included by residual.cu inside namespace tusas, after ElemArgs.
#pragma once

struct Tan3 {
  static const int TX = Tile<3>::X, TY = Tile<3>::Y, TZ = Tile<3>::Z;
  static const int NX = TX + 1, NY = TY + 1, NZ = TZ + 1;
  static const int NT = NX * NY * NZ;  // nodes
  static const int NE = TX * TY * TZ;  // elements = threads
  static const int UX = TX * NY * NZ;  // x-edges
  static const int UY = TX * TY * NZ;  // xy-faces
  // shared-memory layout (doubles): forward buffers, then the transposed ones aliased over them
  static const int OFF_N = 0;                 // [2][NT] staged nodes
  static const int OFF_X = OFF_N + 2 * NT;    // [2][3][UX] x-stage
  static const int OFF_Y = OFF_X + 6 * UX;    // [2][8][UY] y-stage
  static const int FWD = OFF_Y + 16 * UY;
  static const int OFF_ZC = 0;                // [2][2][8][NE] transposed z-stage, per element and level
  static const int OFF_YC = OFF_ZC + 32 * NE; // [2][2][3][UY] transposed y-stage, per face and edge slot
  static const int OFF_XC = 0;                // [2][2][UX] transposed x-stage, per edge and node slot
  static const int BWD = OFF_YC + 12 * UY;
  static const int DOUBLES = FWD > BWD ? FWD : BWD;
  static const size_t BYTES = sizeof(double) * DOUBLES;
};
static_assert(Tan3::BYTES <= 48 * 1024, "tan3_kernel launches without the large-shared-memory opt-in");

template <int MODEL, bool TRANS>
__global__ void __launch_bounds__(Tan3::NE, 3) tan3_kernel(const ElemArgs A) {
  typedef Tan3 G;
  constexpr int TX = G::TX, TY = G::TY, TZ = G::TZ, NX = G::NX, NY = G::NY;
  constexpr int NT = G::NT, NE = G::NE, UX = G::UX, UY = G::UY;
  constexpr int NC = NLin<3, MODEL>::VALUE;
  const double t = TUSAS_GP_T;
  extern __shared__ double sm[];
  double* sN = sm + G::OFF_N;
  double* sX = sm + G::OFF_X;
  double* sY = sm + G::OFF_Y;
  double* sZc = sm + G::OFF_ZC;
  double* sYc = sm + G::OFF_YC;
  double* sXc = sm + G::OFF_XC;

  const DevMesh& m = A.m;
  int b = blockIdx.x;
  const int ix = b % A.ctx;
  b /= A.ctx;
  const int iy = b % A.cty;
  const int iz = b / A.cty;
  const int tile_x = 2 * ix + (A.color & 1);
  const int tile_y = 2 * iy + ((A.color >> 1) & 1);
  const int tile_z = 2 * iz + ((A.color >> 2) & 1);
  const int ex0 = tile_x * TX, ey0 = tile_y * TY, ez0 = tile_z * TZ;
  const int tid = threadIdx.x;

  // ---- A. stage the tile's nodes (zero outside the mesh) ----------------------
  for (int s = tid; s < NT; s += NE) {
    const int lx = s % NX, ly = (s / NX) % NY, lz = s / (NX * NY);
    const int gx = ex0 + lx, gy = ey0 + ly, gz = ez0 + lz;
    const bool ok = gx < m.nnx && gy < m.nny && gz < m.nnz;
    const i64 node = gx + (i64)m.nnx * (gy + (i64)m.nny * gz);
    sN[s] = ok ? A.V[node] : 0.0;
    sN[NT + s] = ok ? A.V[m.nn + node] : 0.0;
  }
  __syncthreads();

  // ---- B. x-stage per x-edge (ex, ny, nz): values at the two x Gauss points, difference
  for (int u = tid; u < UX; u += NE) {
    const int ex = u % TX, r = u / TX;
    const int n0 = ex + NX * r;  // r = ny + NY nz
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double x0 = sN[f * NT + n0], x1 = sN[f * NT + n0 + 1];
      const double bb = x1 - x0;
      sX[(3 * f + 0) * UX + u] = fma(t, bb, x0);
      sX[(3 * f + 1) * UX + u] = fma(-t, bb, x1);
      sX[(3 * f + 2) * UX + u] = bb;
    }
  }
  __syncthreads();

  // ---- C. y-stage per xy-face (ex, ey, nz) from the x-edges at ny = ey, ey + 1:
  // [0..3] values at (x bit, y bit) = k & 1, k >> 1; [4, 5] y-differences at x bit;
  // [6, 7] x-differences at y bit
  for (int u = tid; u < UY; u += NE) {
    const int ex = u % TX, ey = (u / TX) % TY, nz = u / (TX * TY);
    const int lo = ex + TX * (ey + NY * nz), hi = lo + TX;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double* X = sX + 3 * f * UX;
      double* Y = sY + 8 * f * UY;
      {  // x-differences along y first (the order of interp_l)
        const double x0 = X[2 * UX + lo], x1 = X[2 * UX + hi];
        const double bb = x1 - x0;
        Y[6 * UY + u] = fma(t, bb, x0);
        Y[7 * UY + u] = fma(-t, bb, x1);
      }
#pragma unroll
      for (int xb = 0; xb < 2; ++xb) {
        const double x0 = X[xb * UX + lo], x1 = X[xb * UX + hi];
        const double bb = x1 - x0;
        Y[(4 + xb) * UY + u] = bb;
        Y[xb * UY + u] = fma(t, bb, x0);
        Y[(xb + 2) * UY + u] = fma(-t, bb, x1);
      }
    }
  }
  __syncthreads();

  // ---- D. per element: z-stage, pointwise product, transposed z-stage -----------
  const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
  const int ex = ex0 + lx, ey = ey0 + ly, ez = ez0 + lz;
  const bool valid = ex < m.nx && ey < m.ny && ez < m.nz;
  const int uz0 = tid, uz1 = tid + TX * TY;  // faces below and above the element
  double zlo[2][8], zhi[2][8];               // transposed z-stage outputs (face layout)
  if (valid) {
    double val[2][8], grd[2][3][4];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double* Y = sY + 8 * f * UY;
#pragma unroll
      for (int yb = 0; yb < 2; ++yb) {  // x-differences along z: grad[0][y + 2 z]
        const double x0 = Y[(6 + yb) * UY + uz0], x1 = Y[(6 + yb) * UY + uz1];
        const double bb = x1 - x0;
        grd[f][0][yb] = fma(t, bb, x0);
        grd[f][0][yb + 2] = fma(-t, bb, x1);
      }
#pragma unroll
      for (int xb = 0; xb < 2; ++xb) {  // y-differences along z: grad[1][x + 2 z]
        const double x0 = Y[(4 + xb) * UY + uz0], x1 = Y[(4 + xb) * UY + uz1];
        const double bb = x1 - x0;
        grd[f][1][xb] = fma(t, bb, x0);
        grd[f][1][xb + 2] = fma(-t, bb, x1);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // values along z; z-differences grad[2][x + 2 y]
        const double x0 = Y[k * UY + uz0], x1 = Y[k * UY + uz1];
        const double bb = x1 - x0;
        grd[f][2][k] = bb;
        val[f][k] = fma(t, bb, x0);
        val[f][k + 4] = fma(-t, bb, x1);
      }
    }
    const i64 tile_id = tile_x + (i64)A.ntx * (tile_y + (i64)A.nty * tile_z);
    const double* linp = A.lin + tile_id * (i64)(NC * 8 * NE) + tid;  // [c][g][t] within the tile
    double s0[8], s1[8], f0[3][8], f1[3][8];
    GPOut<3> o;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      double L[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) L[c] = __ldg(linp + (c * 8 + g) * NE);
      double xp[3], xg[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        xp[d] = grd[0][d][remove_bit(g, d)];
        xg[d] = grd[1][d][remove_bit(g, d)];
      }
      lin_apply<3, MODEL, TRANS, true>(A.P, L, val[0][g], val[1][g], xp, xg, o, A.K);
      s0[g] = o.sphi;
      s1[g] = o.su;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        f0[d][g] = o.fphi[d];
        f1[d][g] = o.fu[d];
      }
    }
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double* sv = f ? s1 : s0;
      double (*fl)[8] = f ? f1 : f0;
      double F[3][4];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int j = 0; j < 4; ++j) F[d][j] = fl[d][insert_bit(j, d, 0)] + fl[d][insert_bit(j, d, 1)];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // values with the z-differences
        const double yL = sv[k], yR = sv[k + 4];
        const double q = fma(t, yL - yR, F[2][k]);
        zlo[f][k] = yL - q;
        zhi[f][k] = yR + q;
      }
#pragma unroll
      for (int yb = 0; yb < 2; ++yb) {  // x-differences: transposed interpolation along z
        const double yL = F[0][yb], yR = F[0][yb + 2];
        const double dd = yL - yR;
        zlo[f][6 + yb] = fma(-t, dd, yL);
        zhi[f][6 + yb] = fma(t, dd, yR);
      }
#pragma unroll
      for (int xb = 0; xb < 2; ++xb) {  // y-differences
        const double yL = F[1][xb], yR = F[1][xb + 2];
        const double dd = yL - yR;
        zlo[f][4 + xb] = fma(-t, dd, yL);
        zhi[f][4 + xb] = fma(t, dd, yR);
      }
    }
  } else {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
#pragma unroll
      for (int k = 0; k < 8; ++k) zlo[f][k] = zhi[f][k] = 0.0;
    }
  }
  __syncthreads();  // every forward read is done: the transposed buffers alias them
#pragma unroll
  for (int f = 0; f < 2; ++f) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      sZc[((f * 2 + 0) * 8 + k) * NE + tid] = zlo[f][k];
      sZc[((f * 2 + 1) * 8 + k) * NE + tid] = zhi[f][k];
    }
  }
  __syncthreads();

  // ---- E. per face: sum the elements below (upper level) and above (lower level),
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

  // ---- F. per x-edge (ex, ny, nz): sum the faces on both sides in y, transposed x-stage
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

  // ---- G. node sums in fixed order, read-modify-write ---------------------------
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
    }
    const i64 node = gx + (i64)m.nnx * (gy + (i64)m.nny * gz);
    A.out[node] += acc[0];
    A.out[m.nn + node] += acc[1];
  }
}
