// Block-diagonal preconditioner M = diag(M11, M22) of Eq. (pre), blocks of
// Eqs. (pref2) / (preconc2) in Karma-Rappel units:
//   (M11)_ij = (1/dt)(tau0 B(u) a^2 psi_j, psi_i) + theta (W0^2 a^2 grad psi_j, grad psi_i)
//   (M22)_ij = (1/dt)(A(phi^n) psi_j, psi_i)     + theta (D q(phi) grad psi_j, grad psi_i)
// evaluated at the Gauss points of the current Newton iterate, stored as
// 3^dim-point nodal stencils, inverted approximately per block by point
// Jacobi or by one geometric multigrid V-cycle: vertex-centred coarsening by
// 2, (bi/tri)linear prolongation, Galerkin coarse stencils P^T A P, Chebyshev
// smoothing of D^-1 A on [lmax/30, lmax] with lmax the Gershgorin bound
// (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1). The paper
// inverts the blocks with algebraic multigrid and Chebyshev smoothing
// (Sec. 4.4); on the structured box the geometric hierarchy is the natural
// equivalent. Operators, smoother and coarse levels run in FP32 or FP64 (T).
#include <math.h>

#include "precond.h"

namespace tusas {

template <int DIM>
struct Pow3 {
  static const int V = DIM == 2 ? 9 : 27;
};

// ---------------------------------------------------------------------------
// fine-level stencil fill (element tiles, colours, fixed-order node sums)
// ---------------------------------------------------------------------------
template <typename T>
struct FillArgs {
  DevMesh m;
  DevPhys P;
  ScalesT<T> S;
  T theta;
  T w;          // Gauss weight (h/2)^dim
  T ih2;        // 1/h^2
  const double* U;
  const double* Un;
  T* st;        // [2][NS][nn]
  int color, ctx, cty, ctz;
};

template <typename T>
__device__ __forceinline__ T t_rsqrt(T x);
template <>
__device__ __forceinline__ double t_rsqrt<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float t_rsqrt<float>(float x) { return rsqrtf(x); }

// out[p] = sum_g c[g] prod_d tab[d][p_d][g_d]  (p in mixed radix 3, g in radix 2)
template <int DIM, typename T>
__device__ __forceinline__ void contract(const T* c, const T (*tab)[3][2], T* out) {
  T cur[27];
#pragma unroll
  for (int g = 0; g < (1 << DIM); ++g) cur[g] = c[g];
  int p3 = 1;  // 3^d
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    T nxt[27];
    const int nh = 1 << (DIM - d - 1);
#pragma unroll
    for (int pl = 0; pl < 9; ++pl) {
      if (pl >= p3) break;
#pragma unroll
      for (int gh = 0; gh < 4; ++gh) {
        if (gh >= nh) break;
        const T c0 = cur[pl + p3 * (0 + 2 * gh)];
        const T c1 = cur[pl + p3 * (1 + 2 * gh)];
#pragma unroll
        for (int pd = 0; pd < 3; ++pd) nxt[pl + p3 * (pd + 3 * gh)] = c0 * tab[d][pd][0] + c1 * tab[d][pd][1];
      }
    }
    p3 *= 3;
#pragma unroll
    for (int i = 0; i < 27; ++i) cur[i] = nxt[i];
  }
#pragma unroll
  for (int i = 0; i < Pow3<DIM>::V; ++i) out[i] = cur[i];
}

template <int DIM, int MODEL, typename T>
__global__ void __launch_bounds__(Tile<DIM>::X * Tile<DIM>::Y * Tile<DIM>::Z) k_stencil_fill(const FillArgs<T> A) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  constexpr int NX = TX + 1, NY = TY + 1, NZ = DIM == 3 ? TZ + 1 : 1;
  constexpr int NT = NX * NY * NZ;
  constexpr int NE = TX * TY * TZ;
  constexpr int NN = 1 << DIM;
  constexpr int NH = NN / 2;
  constexpr int NS = Pow3<DIM>::V;
  __shared__ T sphi[NT], su[NT], sphin[NT];
  __shared__ T sK[NS][NE];  // element stencil values of one block at a time
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
  for (int s = threadIdx.x; s < NT; s += NE) {
    const int lx = s % NX, ly = (s / NX) % NY, lz = s / (NX * NY);
    const int gx = ex0 + lx, gy = ey0 + ly, gz = ez0 + lz;
    const bool ok = gx < m.nnx && gy < m.nny && gz < m.nnz;
    const i64 node = gx + (i64)m.nnx * (gy + (i64)m.nny * gz);
    sphi[s] = ok ? (T)A.U[node] : T(0);
    su[s] = ok ? (T)A.U[m.nn + node] : T(0);
    sphin[s] = ok ? (T)A.Un[node] : T(0);
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int lx = t % TX, ly = (t / TX) % TY, lz = t / (TX * TY);
  const int ex = ex0 + lx, ey = ey0 + ly, ez = ez0 + lz;
  const bool valid = ex < m.nx && ey < m.ny && (DIM == 2 || ez < m.nz);
  T cmA[NN], ckA[NN], cmB[NN], ckB[NN], tmA[DIM][3][2];
  if (valid) {
    T nphi[NN], nu[NN], npn[NN];
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      const int si = (lx + (a & 1)) + NX * ((ly + ((a >> 1) & 1)) + NY * (lz + ((a >> 2) & 1)));
      nphi[a] = sphi[si];
      nu[a] = su[si];
      npn[a] = sphin[si];
    }
    T phi[NN], u[NN], phin[NN], gp[DIM][NH];
    interp<DIM, true, T>(nphi, phi, gp, A.S);
    interp<DIM, false, T>(nu, u, nullptr, A.S);
    interp<DIM, false, T>(npn, phin, nullptr, A.S);
    T cm1[NN], ck1[NN], cm2[NN], ck2[NN];
    const T eps = (T)A.P.eps4, k = (T)A.P.k;
#pragma unroll
    for (int g = 0; g < NN; ++g) {
      T q = 0, s4 = 0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const T pd = gp[d][remove_bit(g, d)];
        q += pd * pd;
        s4 += pd * pd * pd * pd;
      }
      T a = 1;
      if ((double)q >= TUSAS_GUARD_Q) {
        const T iq = t_rsqrt<T>(q) * t_rsqrt<T>(q);
        a = (T)(1.0 - 3.0 * A.P.eps4) + T(4) * eps * s4 * iq * iq;
      }
      const T a2 = a * a;
      const T B = T(1) + (T(1) - k) * u[g];
      const T Ac = MODEL == 0 ? T(1) : T(0.5) * ((T(1) + k) - (T(1) - k) * phin[g]);
      const T mob = MODEL == 0 ? T(1) : T(0.5) * (T(1) - phi[g]);
      cm1[g] = A.w * (T)A.P.tau0 * B * a2 * (T)A.P.idt;
      ck1[g] = A.w * A.theta * (T)(A.P.W0 * A.P.W0) * a2;
      cm2[g] = A.w * Ac * (T)A.P.idt;
      ck2[g] = A.w * A.theta * (T)A.P.D * mob;
    }
    // 1D tables: mass [p][g] and derivative products [p] (p: 0 = (0,0), 1 = (0,1), 2 = (1,1))
    const T sq = (T)0.57735026918962576;
    const T xi0 = (T(1) - sq) / T(2), xi1 = (T(1) + sq) / T(2);
    T tm[DIM][3][2];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      tm[d][0][0] = (T(1) - xi0) * (T(1) - xi0);
      tm[d][0][1] = (T(1) - xi1) * (T(1) - xi1);
      tm[d][1][0] = xi0 * (T(1) - xi0);
      tm[d][1][1] = xi1 * (T(1) - xi1);
      tm[d][2][0] = xi0 * xi0;
      tm[d][2][1] = xi1 * xi1;
    }
    // element values K[p] per block, p = pair type per axis; stored one block at a time below
#pragma unroll
    for (int g = 0; g < NN; ++g) {
      cmA[g] = cm1[g];
      ckA[g] = ck1[g];
      cmB[g] = cm2[g];
      ckB[g] = ck2[g];
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        tmA[d][p][0] = tm[d][p][0];
        tmA[d][p][1] = tm[d][p][1];
      }
  }
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    if (valid) {
      const T* cm = blk == 0 ? cmA : cmB;
      const T* ck = blk == 0 ? ckA : ckB;
      T K[NS], tmp[NS], tk[DIM][3][2];
      contract<DIM, T>(cm, tmA, K);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
#pragma unroll
        for (int ee = 0; ee < DIM; ++ee) {
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            const T kv = (p == 1 ? -A.ih2 : A.ih2);
            tk[ee][p][0] = ee == d ? kv : tmA[ee][p][0];
            tk[ee][p][1] = ee == d ? kv : tmA[ee][p][1];
          }
        }
        contract<DIM, T>(ck, tk, tmp);
#pragma unroll
        for (int i = 0; i < NS; ++i) K[i] += tmp[i];
      }
#pragma unroll
      for (int i = 0; i < NS; ++i) sK[i][t] = K[i];
    } else {
#pragma unroll
      for (int i = 0; i < NS; ++i) sK[i][t] = T(0);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < NT; s += NE) {
      const int nx_ = s % NX, ny_ = (s / NX) % NY, nz_ = s / (NX * NY);
      const int gx = ex0 + nx_, gy = ey0 + ny_, gz = ez0 + nz_;
      if (gx >= m.nnx || gy >= m.nny || gz >= m.nnz) continue;
      T acc[NS];
#pragma unroll
      for (int o = 0; o < NS; ++o) acc[o] = T(0);
#pragma unroll
      for (int a = 0; a < NN; ++a) {
        const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
        const int elx = nx_ - ax, ely = ny_ - ay, elz = nz_ - az;
        if (elx >= 0 && elx < TX && ely >= 0 && ely < TY && elz >= 0 && elz < TZ) {
          const int e = elx + TX * (ely + TY * elz);
#pragma unroll
          for (int bb = 0; bb < NN; ++bb) {
            const int bx = bb & 1, by = (bb >> 1) & 1, bz = (bb >> 2) & 1;
            const int o = (bx - ax + 1) + 3 * (by - ay + 1) + (DIM == 3 ? 9 * (bz - az + 1) : 0);
            const int p = (ax + bx) + 3 * (ay + by) + (DIM == 3 ? 9 * (az + bz) : 0);
            acc[o] += sK[p][e];
          }
        }
      }
      const i64 node = gx + (i64)m.nnx * (gy + (i64)m.nny * gz);
#pragma unroll
      for (int o = 0; o < NS; ++o) A.st[(blk * NS + o) * m.nn + node] += acc[o];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// stencil helpers
// ---------------------------------------------------------------------------

// Node of the calling thread in a 3D launch (x fastest); false outside the mesh.
__device__ __forceinline__ bool node3(const DevMesh& m, int& ix, int& iy, int& iz, i64& node) {
  ix = blockIdx.x * blockDim.x + threadIdx.x;
  iy = blockIdx.y * blockDim.y + threadIdx.y;
  iz = blockIdx.z * blockDim.z + threadIdx.z;
  if (ix >= m.nnx || iy >= m.nny || iz >= m.nnz) return false;
  node = ix + (i64)m.nnx * (iy + (i64)m.nny * iz);
  return true;
}

// sum_o A[o] x[node + o] in offset order; interior nodes skip the bounds tests
template <int DIM, typename T>
__device__ __forceinline__ T stencil_apply(const T* __restrict__ st, const T* __restrict__ x, const DevMesh& m, i64 node,
                                           int ix, int iy, int iz) {
  constexpr int NS = Pow3<DIM>::V;
  const i64 sy = m.nnx, sz = (i64)m.nnx * m.nny;
  T s = T(0);
  const bool interior = ix > 0 && ix < m.nnx - 1 && iy > 0 && iy < m.nny - 1 && (DIM == 2 || (iz > 0 && iz < m.nnz - 1));
  if (interior) {
#pragma unroll
    for (int o = 0; o < NS; ++o) {
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = DIM == 3 ? o / 9 - 1 : 0;
      const i64 off = ox + sy * oy + sz * oz;
      // symmetric operator: a backward entry A(i, i+o) is read as A(i+o, i), the neighbour's
      // forward entry, so only the 14 forward / centre coefficient arrays are streamed
      const T a = o < NS / 2 ? __ldg(st + (NS - 1 - o) * m.nn + node + off) : __ldg(st + o * m.nn + node);
      s += a * __ldg(x + node + off);
    }
  } else {
#pragma unroll
    for (int o = 0; o < NS; ++o) {
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = DIM == 3 ? o / 9 - 1 : 0;
      const int jx = ix + ox, jy = iy + oy, jz = iz + oz;
      if (jx < 0 || jx >= m.nnx || jy < 0 || jy >= m.nny || jz < 0 || jz >= m.nnz) continue;
      const i64 off = ox + sy * oy + sz * oz;
      const T a = o < NS / 2 ? st[(NS - 1 - o) * m.nn + node + off] : st[o * m.nn + node];
      s += a * x[node + off];
    }
  }
  return s;
}

static dim3 block3(const DevMesh& m) { return m.dim == 3 ? dim3(32, 4, 2) : dim3(32, 8, 1); }
static dim3 grid3(const DevMesh& m) {
  const dim3 b = block3(m);
  return dim3((m.nnx + b.x - 1) / b.x, (m.nny + b.y - 1) / b.y, (m.nnz + b.z - 1) / b.z);
}

static int grid_nodes(i64 n) {
  i64 g = (n + 255) / 256;
  if (g > 148 * 32) g = 148 * 32;
  return (int)(g < 1 ? 1 : g);
}

// Galerkin coarse stencil: A_c(I, J) = sum_{i,j} P(i,I) A(i,j) P(j,J)
template <int DIM, typename T>
__global__ void k_rap(DevMesh mf, DevMesh mc, const T* __restrict__ stf, T* __restrict__ stc) {
  constexpr int NS = Pow3<DIM>::V;
  {
    int cx, cy, cz;
    i64 I;
    if (!node3(mc, cx, cy, cz, I)) return;
    for (int blk = 0; blk < 2; ++blk) {
      T acc[NS];
#pragma unroll
      for (int o = 0; o < NS; ++o) acc[o] = T(0);
      for (int o1 = 0; o1 < NS; ++o1) {
        const int o1x = o1 % 3 - 1, o1y = (o1 / 3) % 3 - 1, o1z = DIM == 3 ? o1 / 9 - 1 : 0;
        const int fx = 2 * cx + o1x, fy = 2 * cy + o1y, fz = 2 * cz + o1z;
        if (fx < 0 || fx >= mf.nnx || fy < 0 || fy >= mf.nny || fz < 0 || fz >= mf.nnz) continue;
        const T w1 = (o1x ? T(0.5) : T(1)) * (o1y ? T(0.5) : T(1)) * (o1z ? T(0.5) : T(1));
        const i64 fi = fx + (i64)mf.nnx * (fy + (i64)mf.nny * fz);
#pragma unroll
        for (int o2 = 0; o2 < NS; ++o2) {
          const T av = stf[(blk * NS + o2) * mf.nn + fi];
          if (av == T(0)) continue;
          const int o2x = o2 % 3 - 1, o2y = (o2 / 3) % 3 - 1, o2z = DIM == 3 ? o2 / 9 - 1 : 0;
          const int r[3] = {o1x + o2x, o1y + o2y, o1z + o2z};
          int lo[3], hi[3];
          T wl[3], wh[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            if ((r[d] & 1) == 0) {
              lo[d] = hi[d] = r[d] / 2;
              wl[d] = T(1);
              wh[d] = T(0);
            } else {
              lo[d] = (r[d] - 1) / 2;
              hi[d] = (r[d] + 1) / 2;
              wl[d] = wh[d] = T(0.5);
            }
          }
          const T v = w1 * av;
#pragma unroll
          for (int c = 0; c < (1 << DIM); ++c) {
            const T wx = (c & 1) ? wh[0] : wl[0];
            const T wy = (c & 2) ? wh[1] : wl[1];
            const T wz = DIM == 3 ? ((c & 4) ? wh[2] : wl[2]) : T(1);
            const T ww = wx * wy * wz;
            if (ww == T(0)) continue;
            const int jx = (c & 1) ? hi[0] : lo[0], jy = (c & 2) ? hi[1] : lo[1];
            const int jz = DIM == 3 ? ((c & 4) ? hi[2] : lo[2]) : 0;
            const int oc = (jx + 1) + 3 * (jy + 1) + (DIM == 3 ? 9 * (jz + 1) : 0);
            acc[oc] += v * ww;
          }
        }
      }
#pragma unroll
      for (int o = 0; o < NS; ++o) stc[(blk * NS + o) * mc.nn + I] = acc[o];
    }
  }
}

// D^-1 and the Gershgorin bound max_i sum_j |a_ij| / a_ii per block.
template <int DIM, typename T>
__global__ void k_gersh(DevMesh m, const T* __restrict__ st, T* __restrict__ dinv, double* __restrict__ partials) {
  constexpr int NS = Pow3<DIM>::V;
  constexpr int C = NS / 2;
  __shared__ double red[2][256];
  double mx[2] = {0.0, 0.0};
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < m.nn; i += (i64)gridDim.x * blockDim.x) {
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      double s = 0.0;
#pragma unroll
      for (int o = 0; o < NS; ++o) s += fabs((double)st[(blk * NS + o) * m.nn + i]);
      const double c = (double)st[(blk * NS + C) * m.nn + i];
      dinv[blk * m.nn + i] = (T)(1.0 / c);
      mx[blk] = fmax(mx[blk], s / c);
    }
  }
  red[0][threadIdx.x] = mx[0];
  red[1][threadIdx.x] = mx[1];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + w]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = red[0][0];
    partials[2 * blockIdx.x + 1] = red[1][0];
  }
}

__global__ void k_max_partials(int nb, const double* __restrict__ partials, double* __restrict__ out) {
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v = fmax(v, partials[2 * b + threadIdx.x]);
    out[threadIdx.x] = v;
  }
}

// ---------------------------------------------------------------------------
// Chebyshev smoother, residual, transfers
// ---------------------------------------------------------------------------
template <typename T>
struct Coef2 {
  T a[2], b[2];
};

// r = D^-1 (b - A x) (or D^-1 b if x == nullptr, and then x = 0); d = r * it
template <int DIM, typename T>
__global__ void k_cheb_init(DevMesh m, const T* __restrict__ st, const T* __restrict__ dinv, const T* __restrict__ bvec,
                            T* __restrict__ x, int zero_x, T* __restrict__ r, T* __restrict__ d, Coef2<T> it) {
  constexpr int NS = Pow3<DIM>::V;
  {
    int ix, iy, iz;
    i64 i;
    if (!node3(m, ix, iy, iz, i)) return;
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      T v = bvec[blk * m.nn + i];
      if (zero_x)
        x[blk * m.nn + i] = T(0);
      else
        v -= stencil_apply<DIM, T>(st + blk * NS * m.nn, x + blk * m.nn, m, i, ix, iy, iz);
      const T rr = dinv[blk * m.nn + i] * v;
      r[blk * m.nn + i] = rr;
      d[blk * m.nn + i] = rr * it.a[blk];
    }
  }
}

// x += d; if !last: r -= D^-1 A d; dout = c1 d + c2 r
template <int DIM, typename T>
__global__ void k_cheb_step(DevMesh m, const T* __restrict__ st, const T* __restrict__ dinv, T* __restrict__ x,
                            T* __restrict__ r, const T* __restrict__ d, T* __restrict__ dout, Coef2<T> c, int last) {
  constexpr int NS = Pow3<DIM>::V;
  {
    int ix, iy, iz;
    i64 i;
    if (!node3(m, ix, iy, iz, i)) return;
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      const i64 k = blk * m.nn + i;
      const T dk = d[k];
      x[k] += dk;
      if (!last) {
        const T ad = stencil_apply<DIM, T>(st + blk * NS * m.nn, d + blk * m.nn, m, i, ix, iy, iz);
        const T rr = r[k] - dinv[k] * ad;
        r[k] = rr;
        dout[k] = c.a[blk] * dk + c.b[blk] * rr;
      }
    }
  }
}

template <int DIM, typename T>
__global__ void k_resid(DevMesh m, const T* __restrict__ st, const T* __restrict__ bvec, const T* __restrict__ x,
                        T* __restrict__ res) {
  constexpr int NS = Pow3<DIM>::V;
  {
    int ix, iy, iz;
    i64 i;
    if (!node3(m, ix, iy, iz, i)) return;
#pragma unroll
    for (int blk = 0; blk < 2; ++blk)
      res[blk * m.nn + i] =
          bvec[blk * m.nn + i] - stencil_apply<DIM, T>(st + blk * NS * m.nn, x + blk * m.nn, m, i, ix, iy, iz);
  }
}

// b_c(I) = sum_i P(i, I) res(i) over the fine nodes within distance 1 of 2I
template <int DIM, typename T>
__global__ void k_restrict(DevMesh mf, DevMesh mc, const T* __restrict__ res, T* __restrict__ bc) {
  constexpr int NS = Pow3<DIM>::V;
  {
    int cx, cy, cz;
    i64 I;
    if (!node3(mc, cx, cy, cz, I)) return;
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      T s = T(0);
#pragma unroll
      for (int o = 0; o < NS; ++o) {
        const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = DIM == 3 ? o / 9 - 1 : 0;
        const int fx = 2 * cx + ox, fy = 2 * cy + oy, fz = 2 * cz + oz;
        if (fx < 0 || fx >= mf.nnx || fy < 0 || fy >= mf.nny || fz < 0 || fz >= mf.nnz) continue;
        const T w = (ox ? T(0.5) : T(1)) * (oy ? T(0.5) : T(1)) * (oz ? T(0.5) : T(1));
        s += w * res[blk * mf.nn + fx + (i64)mf.nnx * (fy + (i64)mf.nny * fz)];
      }
      bc[blk * mc.nn + I] = s;
    }
  }
}

// x_f(i) += sum_J P(i, J) x_c(J)
template <int DIM, typename T>
__global__ void k_prolong(DevMesh mf, DevMesh mc, const T* __restrict__ xc, T* __restrict__ xf) {
  {
    int fx, fy, fz;
    i64 i;
    if (!node3(mf, fx, fy, fz, i)) return;
    const int f[3] = {fx, fy, fz};
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      T s = T(0);
#pragma unroll
      for (int c = 0; c < (1 << DIM); ++c) {
        int J[3] = {0, 0, 0};
        T w = T(1);
        bool ok = true;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const int hi = (c >> d) & 1;
          if ((f[d] & 1) == 0) {
            if (hi) ok = false;
            J[d] = f[d] / 2;
          } else {
            J[d] = f[d] / 2 + hi;
            w *= T(0.5);
          }
        }
        if (!ok) continue;
        s += w * xc[blk * mc.nn + J[0] + (i64)mc.nnx * (J[1] + (i64)mc.nny * J[2])];
      }
      xf[blk * mf.nn + i] += s;
    }
  }
}

template <typename T>
__global__ void k_to_t(i64 n, const double* __restrict__ r, T* __restrict__ b) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) b[i] = (T)r[i];
}
template <typename T>
__global__ void k_from_t(i64 n, const T* __restrict__ x, double* __restrict__ z) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) z[i] = (double)x[i];
}
template <typename T>
__global__ void k_recip(i64 n, const double* __restrict__ d, T* __restrict__ dinv) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    dinv[i] = (T)(1.0 / d[i]);
}
template <typename T>
__global__ void k_jacobi(i64 n, const T* __restrict__ dinv, const double* __restrict__ r, double* __restrict__ z) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    z[i] = (double)dinv[i] * r[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static DevMesh coarsen(const DevMesh& m) {
  DevMesh c = m;
  c.nx = m.nx / 2;
  c.ny = m.ny / 2;
  c.nz = m.dim == 3 ? m.nz / 2 : 0;
  c.nnx = c.nx + 1;
  c.nny = c.ny + 1;
  c.nnz = m.dim == 3 ? c.nz + 1 : 1;
  c.nn = (i64)c.nnx * c.nny * c.nnz;
  c.ne = (i64)c.nx * c.ny * (m.dim == 3 ? c.nz : 1);
  c.h = 2 * m.h;
  return c;
}
static bool can_coarsen(const DevMesh& m) {
  bool ok = m.nx % 2 == 0 && m.ny % 2 == 0 && m.nx >= 2 && m.ny >= 2;
  if (m.dim == 3) ok = ok && m.nz % 2 == 0 && m.nz >= 2;
  return ok;
}

cudaError_t Precond::create(const DevMesh& m, int kind_, int fp32_, int levels, int cheb_degree_, int coarse_degree_) {
  kind = kind_;
  fp32 = fp32_;
  cheb_degree = cheb_degree_;
  coarse_degree = coarse_degree_;
  lv.clear();
  bytes = 0;
  if (kind == 0) return cudaSuccess;
  const size_t esz = fp32 ? sizeof(float) : sizeof(double);
  if (m.order == 2) {
    if (kind != 1) return cudaErrorInvalidValue;
    PrecondLevel L = {};
    L.m = m;
    L.nn = m.nn;
    cudaError_t e = cudaMalloc(&L.dinv, esz * 2 * m.nn);
    if (e != cudaSuccess) return e;
    lv.push_back(L);
    bytes += (esz + sizeof(double)) * 2 * m.nn;
    return cudaMalloc(&diag, sizeof(double) * 2 * m.nn);
  }
  const int NS = m.dim == 3 ? 27 : 9;
  const int nlev = kind == 1 ? 1 : (levels < 1 ? 1 : levels);
  DevMesh cur = m;
  for (int l = 0; l < nlev; ++l) {
    PrecondLevel L = {};
    L.m = cur;
    L.nn = cur.nn;
    void** bufs[] = {&L.dinv, &L.b, &L.x, &L.r, &L.d, &L.d2, &L.res};
    cudaError_t e = cudaMalloc(&L.st, esz * 2 * NS * cur.nn);
    if (e != cudaSuccess) return e;
    bytes += esz * 2 * NS * cur.nn;
    const int nvec = kind == 1 ? 1 : 7;
    for (int v = 0; v < nvec; ++v) {
      e = cudaMalloc(bufs[v], esz * 2 * cur.nn);
      if (e != cudaSuccess) return e;
      bytes += esz * 2 * cur.nn;
    }
    lv.push_back(L);
    if (!can_coarsen(cur)) break;
    cur = coarsen(cur);
  }
  cudaError_t e = cudaMalloc(&gersh_partials, sizeof(double) * 2 * 148 * 32);
  if (e != cudaSuccess) return e;
  return cudaMalloc(&lmax_dev, sizeof(double) * 2 * lv.size());
}

void Precond::destroy() {
  for (auto& L : lv) {
    void* bufs[] = {L.st, L.dinv, L.b, L.x, L.r, L.d, L.d2, L.res};
    for (void* p : bufs)
      if (p) cudaFree(p);
  }
  lv.clear();
  if (gersh_partials) cudaFree(gersh_partials);
  if (lmax_dev) cudaFree(lmax_dev);
  if (diag) cudaFree(diag);
  gersh_partials = lmax_dev = diag = nullptr;
}

template <typename T>
cudaError_t Precond::setup_t(const ElemCtx& c, double theta, const double* U, const double* Un, cudaStream_t st) {
  const DevMesh& m = c.m;
  const int NS = m.dim == 3 ? 27 : 9;
  PrecondLevel& L0 = lv[0];
  if (m.order == 2) {
    // point Jacobi: element pass for diag(M11), diag(M22), then the reciprocals
    cudaError_t e = elem_run(M_DIAG, c, U, Un, nullptr, diag, nullptr, st);
    if (e != cudaSuccess) return e;
    k_recip<T><<<grid_nodes(2 * m.nn), 256, 0, st>>>(2 * m.nn, diag, (T*)L0.dinv);
    count_launches(1);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(L0.st, 0, sizeof(T) * 2 * NS * m.nn, st);
  if (e != cudaSuccess) return e;
  FillArgs<T> A;
  A.m = m;
  A.P = c.P;
  for (int k = 0; k < 4; ++k) {
    A.S.vs[k] = (T)c.S.vs[k];
    A.S.vsw[k] = (T)c.S.vsw[k];
  }
  for (int k = 0; k < 3; ++k) {
    A.S.gs[k] = (T)c.S.gs[k];
    A.S.gsw[k] = (T)c.S.gsw[k];
  }
  A.theta = (T)theta;
  A.w = (T)(m.dim == 3 ? pow(m.h / 2, 3) : pow(m.h / 2, 2));
  A.ih2 = (T)(1.0 / (m.h * m.h));
  A.U = U;
  A.Un = Un;
  A.st = (T*)L0.st;
  const int ntx = c.ntx, nty = c.nty, ntz = c.ntz;
  for (int col = 0; col < (1 << m.dim); ++col) {
    const int cx = col & 1, cy = (col >> 1) & 1, cz = (col >> 2) & 1;
    A.color = col;
    A.ctx = (ntx - cx + 1) / 2;
    A.cty = (nty - cy + 1) / 2;
    A.ctz = m.dim == 3 ? (ntz - cz + 1) / 2 : 1;
    const long long blocks = (long long)A.ctx * A.cty * A.ctz;
    if (blocks <= 0) continue;
    if (m.dim == 3) {
      if (c.P.model == 0)
        {
          k_stencil_fill<3, 0, T><<<(unsigned)blocks, 128, 0, st>>>(A);
          count_launches(1);
        }
      else
        {
          k_stencil_fill<3, 1, T><<<(unsigned)blocks, 128, 0, st>>>(A);
          count_launches(1);
        }
    } else {
      if (c.P.model == 0)
        {
          k_stencil_fill<2, 0, T><<<(unsigned)blocks, 128, 0, st>>>(A);
          count_launches(1);
        }
      else
        {
          k_stencil_fill<2, 1, T><<<(unsigned)blocks, 128, 0, st>>>(A);
          count_launches(1);
        }
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (size_t l = 1; l < lv.size(); ++l) {
    if (m.dim == 3)
      {
        k_rap<3, T><<<grid3(lv[l].m), block3(lv[l].m), 0, st>>>(lv[l - 1].m, lv[l].m, (const T*)lv[l - 1].st, (T*)lv[l].st);
        count_launches(1);
      }
    else
      {
        k_rap<2, T><<<grid3(lv[l].m), block3(lv[l].m), 0, st>>>(lv[l - 1].m, lv[l].m, (const T*)lv[l - 1].st, (T*)lv[l].st);
        count_launches(1);
      }
  }
  for (size_t l = 0; l < lv.size(); ++l) {
    const int nb = grid_nodes(lv[l].nn);
    if (m.dim == 3)
      {
        k_gersh<3, T><<<nb, 256, 0, st>>>(lv[l].m, (const T*)lv[l].st, (T*)lv[l].dinv, gersh_partials);
        count_launches(1);
      }
    else
      {
        k_gersh<2, T><<<nb, 256, 0, st>>>(lv[l].m, (const T*)lv[l].st, (T*)lv[l].dinv, gersh_partials);
        count_launches(1);
      }
    {
      k_max_partials<<<1, 32, 0, st>>>(nb, gersh_partials, lmax_dev + 2 * l);
      count_launches(1);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  std::vector<double> lm(2 * lv.size());
  e = cudaMemcpyAsync(lm.data(), lmax_dev, sizeof(double) * lm.size(), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (size_t l = 0; l < lv.size(); ++l) {
    lv[l].lmax[0] = lm[2 * l];
    lv[l].lmax[1] = lm[2 * l + 1];
  }
  return cudaSuccess;
}

cudaError_t Precond::setup(const ElemCtx& c, double theta, const double* U, const double* Un, cudaStream_t st) {
  if (kind == 0) return cudaSuccess;
  return fp32 ? setup_t<float>(c, theta, U, Un, st) : setup_t<double>(c, theta, U, Un, st);
}

template <typename T>
cudaError_t Precond::cheb(int l, bool zero_x, int degree, cudaStream_t st) {
  PrecondLevel& L = lv[l];
  Coef2<T> it, cc;
  double theta[2], delta[2], sigma[2], rho[2];
  for (int b = 0; b < 2; ++b) {
    const double hi = L.lmax[b], lo = hi / 30.0;
    theta[b] = 0.5 * (hi + lo);
    delta[b] = 0.5 * (hi - lo);
    sigma[b] = theta[b] / delta[b];
    rho[b] = 1.0 / sigma[b];
    it.a[b] = (T)(1.0 / theta[b]);
    it.b[b] = T(0);
  }
  const bool d3 = L.m.dim == 3;
  if (d3)
    {
      k_cheb_init<3, T><<<grid3(L.m), block3(L.m), 0, st>>>(L.m, (const T*)L.st, (const T*)L.dinv, (const T*)L.b, (T*)L.x, zero_x,
                                           (T*)L.r, (T*)L.d, it);
      count_launches(1);
    }
  else
    {
      k_cheb_init<2, T><<<grid3(L.m), block3(L.m), 0, st>>>(L.m, (const T*)L.st, (const T*)L.dinv, (const T*)L.b, (T*)L.x, zero_x,
                                           (T*)L.r, (T*)L.d, it);
      count_launches(1);
    }
  T* dcur = (T*)L.d;
  T* dnext = (T*)L.d2;
  for (int kk = 0; kk < degree; ++kk) {
    const int last = kk == degree - 1;
    for (int b = 0; b < 2; ++b) {
      const double rn = 1.0 / (2.0 * sigma[b] - rho[b]);
      cc.a[b] = (T)(rn * rho[b]);
      cc.b[b] = (T)(2.0 * rn / delta[b]);
      rho[b] = rn;
    }
    if (d3)
      {
        k_cheb_step<3, T><<<grid3(L.m), block3(L.m), 0, st>>>(L.m, (const T*)L.st, (const T*)L.dinv, (T*)L.x, (T*)L.r, dcur, dnext, cc,
                                             last);
        count_launches(1);
      }
    else
      {
        k_cheb_step<2, T><<<grid3(L.m), block3(L.m), 0, st>>>(L.m, (const T*)L.st, (const T*)L.dinv, (T*)L.x, (T*)L.r, dcur, dnext, cc,
                                             last);
        count_launches(1);
      }
    T* tmp = dcur;
    dcur = dnext;
    dnext = tmp;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t Precond::vcycle(int l, cudaStream_t st) {
  const int last = (int)lv.size() - 1;
  if (l == last) return cheb<T>(l, true, coarse_degree, st);
  cudaError_t e = cheb<T>(l, true, cheb_degree, st);
  if (e != cudaSuccess) return e;
  PrecondLevel& F = lv[l];
  PrecondLevel& C = lv[l + 1];
  const bool d3 = F.m.dim == 3;
  if (d3) {
    {
      k_resid<3, T><<<grid3(F.m), block3(F.m), 0, st>>>(F.m, (const T*)F.st, (const T*)F.b, (const T*)F.x, (T*)F.res);
      count_launches(1);
    }
    {
      k_restrict<3, T><<<grid3(C.m), block3(C.m), 0, st>>>(F.m, C.m, (const T*)F.res, (T*)C.b);
      count_launches(1);
    }
  } else {
    {
      k_resid<2, T><<<grid3(F.m), block3(F.m), 0, st>>>(F.m, (const T*)F.st, (const T*)F.b, (const T*)F.x, (T*)F.res);
      count_launches(1);
    }
    {
      k_restrict<2, T><<<grid3(C.m), block3(C.m), 0, st>>>(F.m, C.m, (const T*)F.res, (T*)C.b);
      count_launches(1);
    }
  }
  e = vcycle<T>(l + 1, st);
  if (e != cudaSuccess) return e;
  if (d3)
    {
      k_prolong<3, T><<<grid3(F.m), block3(F.m), 0, st>>>(F.m, C.m, (const T*)C.x, (T*)F.x);
      count_launches(1);
    }
  else
    {
      k_prolong<2, T><<<grid3(F.m), block3(F.m), 0, st>>>(F.m, C.m, (const T*)C.x, (T*)F.x);
      count_launches(1);
    }
  return cheb<T>(l, false, cheb_degree, st);
}

template <typename T>
cudaError_t Precond::apply_t(const double* r, double* z, cudaStream_t st) {
  PrecondLevel& L0 = lv[0];
  const i64 n = 2 * L0.nn;
  if (kind == 1) {
    {
      k_jacobi<T><<<grid_nodes(n), 256, 0, st>>>(n, (const T*)L0.dinv, r, z);
      count_launches(1);
    }
    return cudaGetLastError();
  }
  {
    k_to_t<T><<<grid_nodes(n), 256, 0, st>>>(n, r, (T*)L0.b);
    count_launches(1);
  }
  cudaError_t e = vcycle<T>(0, st);
  if (e != cudaSuccess) return e;
  {
    k_from_t<T><<<grid_nodes(n), 256, 0, st>>>(n, (const T*)L0.x, z);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t Precond::apply(const double* r, double* z, cudaStream_t st) {
  if (kind == 0) {
    if (lv.empty()) return cudaErrorInvalidValue;
    return cudaErrorInvalidValue;
  }
  return fp32 ? apply_t<float>(r, z, st) : apply_t<double>(r, z, st);
}

}  // namespace tusas
