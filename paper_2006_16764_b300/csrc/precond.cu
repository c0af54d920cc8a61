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
// On a Q2 box the finest level is its node grid seen as a box of spacing h/2
// (25-point stencils); its Galerkin coarsening is the grid of element vertices.
#include <math.h>

#include <utility>

#include "precond.h"

namespace tusas {

template <int DIM>
struct Pow3 {
  static const int V = DIM == 2 ? 9 : 27;
};
// stencil of radius R: (2R + 1)^dim entries (R = 2 only on the Q2 node lattice)
template <int DIM, int R>
struct Sten {
  static const int W = 2 * R + 1;
  static const int V = DIM == 2 ? W * W : W * W * W;
};

// ---------------------------------------------------------------------------
// fine-level stencil fill
//
// Node-centric gather: a CTA owns a box of nodes (FillTile), first computes
// the 3^dim "pair-type" element values of both blocks for every element
// touching the box (shared memory), then each thread sums the contributions of
// its <= 2^dim elements in a fixed order and writes its full stencil rows once.
// Elements on the box boundary are evaluated by both neighbouring CTAs (FP32
// work, cheap); every stencil entry is written exactly once, without a
// read-modify-write, so no colouring is needed and the result is deterministic.
// ---------------------------------------------------------------------------
template <typename T>
struct FillArgs {
  DevMesh m;
  DevPhys P;
  ScalesT<T> S;
  T theta;
  T w;          // Gauss weight (h/2)^dim
  T ih2;        // 1/h^2
  // Gauss-point constants in the fill precision (host-computed, so that an FP32 fill does no
  // FP64 arithmetic per Gauss point): small-gradient guard, 1 - 3 eps4, 4 eps4, 1 - k,
  // (1 + k)/2, (1 - k)/2, and the weights of the four coefficients w tau0/dt, w theta W0^2,
  // w/dt, w theta D
  T guard, one_m3e, four_e, omk, half_opk, half_omk, wm1, wk1, wm2, wk2;
  const double* U;
  const double* Un;
  T* st;        // [2][NS][nn]
};

// node box of one CTA, one thread per node (256 threads; the 3D FP64 variant halves x, 128
// threads, to fit its element values in shared memory)
template <int DIM, typename T>
struct FillTile {
  static const int X = (DIM == 3 && sizeof(T) == 8) ? 16 : 32;
  static const int Y = DIM == 3 ? 4 : 8;
  static const int Z = DIM == 3 ? 2 : 1;
  static const int EX = X + 1, EY = Y + 1, EZ = DIM == 3 ? Z + 1 : 1;  // element box
  static const int NEL = EX * EY * EZ;
  static const int THREADS = X * Y * Z;
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

// Pair-type values K[blk][p] of element (ex, ey, ez): the element matrix entry of local
// nodes (a, b) is K[blk][p] with p_d = a_d + b_d per axis (the 1D mass and stiffness
// factors are symmetric in a_d, b_d). Gauss-point coefficients of Eqs. (pref2), (preconc2).
template <int DIM, int MODEL, typename T>
__device__ __forceinline__ void elem_pair_values(const FillArgs<T>& A, int ex, int ey, int ez, T* K0, T* K1) {
  constexpr int NN = 1 << DIM;
  constexpr int NH = NN / 2;
  constexpr int NS = Pow3<DIM>::V;
  const DevMesh& m = A.m;
  T nphi[NN], nu[NN], npn[NN];
#pragma unroll
  for (int a = 0; a < NN; ++a) {
    const i64 node = (ex + (a & 1)) + (i64)m.nnx * ((ey + ((a >> 1) & 1)) + (i64)m.nny * (ez + ((a >> 2) & 1)));
    nphi[a] = narrow<T>(__ldg(A.U + node));
    nu[a] = narrow<T>(__ldg(A.U + m.nn + node));
    npn[a] = narrow<T>(__ldg(A.Un + node));
  }
  T phi[NN], u[NN], phin[NN], gp[DIM][NH];
  interp<DIM, true, T>(nphi, phi, gp, A.S);
  interp<DIM, false, T>(nu, u, nullptr, A.S);
  interp<DIM, false, T>(npn, phin, nullptr, A.S);
  T cm1[NN], ck1[NN], cm2[NN], ck2[NN];
#pragma unroll
  for (int g = 0; g < NN; ++g) {
    T q = 0, s4 = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const T pd = gp[d][remove_bit(g, d)];
      const T pd2 = pd * pd;
      q += pd2;
      s4 += pd2 * pd2;
    }
    T a = 1;
    if (q >= A.guard) {
      const T r = t_rsqrt<T>(q);
      const T iq = r * r;
      a = A.one_m3e + A.four_e * s4 * iq * iq;
    }
    const T a2 = a * a;
    const T B = T(1) + A.omk * u[g];
    const T Ac = MODEL == 0 ? T(1) : A.half_opk - A.half_omk * phin[g];
    const T mob = MODEL == 0 ? T(1) : T(0.5) * (T(1) - phi[g]);
    cm1[g] = A.wm1 * B * a2;
    ck1[g] = A.wk1 * a2;
    cm2[g] = A.wm2 * Ac;
    ck2[g] = A.wk2 * mob;
  }
  // 1D tables: mass [p][g] (p: 0 = (0,0), 1 = (0,1), 2 = (1,1)); stiffness +-1/h^2
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
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    const T* cm = blk == 0 ? cm1 : cm2;
    const T* ck = blk == 0 ? ck1 : ck2;
    T* K = blk == 0 ? K0 : K1;
    T tmp[NS], tk[DIM][3][2];
    contract<DIM, T>(cm, tm, K);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
      for (int ee = 0; ee < DIM; ++ee) {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const T kv = (p == 1 ? -A.ih2 : A.ih2);
          tk[ee][p][0] = ee == d ? kv : tm[ee][p][0];
          tk[ee][p][1] = ee == d ? kv : tm[ee][p][1];
        }
      }
      contract<DIM, T>(ck, tk, tmp);
#pragma unroll
      for (int i = 0; i < NS; ++i) K[i] += tmp[i];
    }
  }
}

template <int DIM, int MODEL, typename T>
__global__ void __launch_bounds__(256) k_stencil_fill(const FillArgs<T> A) {
  using FT = FillTile<DIM, T>;
  constexpr int NN = 1 << DIM;
  constexpr int NS = Pow3<DIM>::V;
  constexpr int NEL = FT::NEL;
  extern __shared__ __align__(16) unsigned char fill_smem[];
  T* sK = reinterpret_cast<T*>(fill_smem);  // [2 NS][NEL]
  const DevMesh& m = A.m;
  const int nx0 = blockIdx.x * FT::X, ny0 = blockIdx.y * FT::Y, nz0 = blockIdx.z * FT::Z;
  // element box: elements nx0 - 1 .. nx0 + X - 1 per axis (those touching the node box)
  for (int le = threadIdx.x; le < NEL; le += blockDim.x) {
    const int lx = le % FT::EX, ly = (le / FT::EX) % FT::EY, lz = le / (FT::EX * FT::EY);
    const int ex = nx0 - 1 + lx, ey = ny0 - 1 + ly, ez = DIM == 3 ? nz0 - 1 + lz : 0;
    const bool ok = ex >= 0 && ex < m.nx && ey >= 0 && ey < m.ny && (DIM == 2 || (ez >= 0 && ez < m.nz));
    T K0[NS], K1[NS];
    if (ok) {
      elem_pair_values<DIM, MODEL, T>(A, ex, ey, ez, K0, K1);
    } else {
#pragma unroll
      for (int i = 0; i < NS; ++i) K0[i] = K1[i] = T(0);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      sK[i * NEL + le] = K0[i];
      sK[(NS + i) * NEL + le] = K1[i];
    }
  }
  __syncthreads();
  const int tx = threadIdx.x % FT::X, ty = (threadIdx.x / FT::X) % FT::Y, tz = threadIdx.x / (FT::X * FT::Y);
  const int ix = nx0 + tx, iy = ny0 + ty, iz = nz0 + tz;
  if (ix >= m.nnx || iy >= m.nny || iz >= m.nnz) return;
  const i64 node = ix + (i64)m.nnx * (iy + (i64)m.nny * iz);
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    T acc[NS];
#pragma unroll
    for (int o = 0; o < NS; ++o) acc[o] = T(0);
    // element with local node a = (ax, ay, az) at this node sits at element-box index
    // (tx + 1 - ax, ty + 1 - ay, tz + 1 - az); out-of-mesh elements hold zeros
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
      const int le = (tx + 1 - ax) + FT::EX * ((ty + 1 - ay) + FT::EY * (DIM == 3 ? tz + 1 - az : 0));
#pragma unroll
      for (int bb = 0; bb < NN; ++bb) {
        const int bx = bb & 1, by = (bb >> 1) & 1, bz = (bb >> 2) & 1;
        const int o = (bx - ax + 1) + 3 * (by - ay + 1) + (DIM == 3 ? 9 * (bz - az + 1) : 0);
        const int p = (ax + bx) + 3 * (ay + by) + (DIM == 3 ? 9 * (az + bz) : 0);
        acc[o] += sK[(blk * NS + p) * NEL + le];
      }
    }
#pragma unroll
    for (int o = 0; o < NS; ++o) A.st[(blk * NS + o) * m.nn + node] = acc[o];
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

// Node and block (M11 / M22) of the calling thread in a smoother launch: the grid's z
// extent is twice the node grid's, blocks one after the other (grid3b).
__device__ __forceinline__ bool node3b(const DevMesh& m, int& ix, int& iy, int& iz, i64& node, int& blk) {
  const int zb = gridDim.z >> 1;
  blk = blockIdx.z >= zb;
  ix = blockIdx.x * blockDim.x + threadIdx.x;
  iy = blockIdx.y * blockDim.y + threadIdx.y;
  iz = (blockIdx.z - blk * zb) * blockDim.z + threadIdx.z;
  if (ix >= m.nnx || iy >= m.nny || iz >= m.nnz) return false;
  node = ix + (i64)m.nnx * (iy + (i64)m.nny * iz);
  return true;
}

// 27-point sum of a 3D radius-1 stencil with 32-bit offsets from the node (for levels whose
// 27 x nn coefficient index fits an int). Used for every node whose y and z neighbours exist
// (fast27), including the first and last node of an x-row: there the x-neighbour index wraps
// to the adjacent row, a valid address whose coefficient is exactly zero (the fine fill and
// the Galerkin products give zero entries towards nodes outside the box), so the product adds
// +0 and the sum is that of the generic loop. Only rows on a y or z face take the loop with
// bounds tests, so warps along x no longer run both paths.
// Whether every neighbour index node + ox + sy oy + sz oz (|o| <= 1) lies in [0, nn): y and z
// neighbours exist, and the two extreme offsets stay inside the array (they fail only at the
// first and last node of the box's second / second-to-last row and layer).
__device__ __forceinline__ bool fast27(const DevMesh& m, int iy, int iz, i64 node, i64 sy, i64 sz) {
  return iy >= 1 && iy < m.nny - 1 && iz >= 1 && iz < m.nnz - 1 && node - 1 - sy - sz >= 0 &&
         node + 1 + sy + sz < m.nn && m.nn * 27 < (i64)0x7fffffff;
}

template <typename T, typename V>
__device__ __forceinline__ T stencil27_i32(const T* __restrict__ st, int nn, int node, int sy, int sz, V val) {
  const T* sp = st + node;
  T s = T(0);
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
    const int off = ox + sy * oy + sz * oz;
    const T a = o < 13 ? __ldg(sp + ((26 - o) * nn + off)) : __ldg(sp + o * nn);
    s += a * val(off);
  }
  return s;
}

// sum_o A[o] x[node + o] in offset order; interior nodes skip the bounds tests
template <int DIM, typename T, int R = 1>
__device__ __forceinline__ T stencil_apply(const T* __restrict__ st, const T* __restrict__ x, const DevMesh& m, i64 node,
                                           int ix, int iy, int iz) {
  constexpr int NS = Sten<DIM, R>::V, W = Sten<DIM, R>::W;
  const i64 sy = m.nnx, sz = (i64)m.nnx * m.nny;
  T s = T(0);
  const bool interior = ix >= R && ix < m.nnx - R && iy >= R && iy < m.nny - R &&
                        (DIM == 2 || (iz >= R && iz < m.nnz - R));
  if (DIM == 3 && R == 1 && fast27(m, iy, iz, node, sy, sz)) {
    const T* xp = x + node;
    return stencil27_i32<T>(st, (int)m.nn, (int)node, (int)sy, (int)sz, [&](int off) { return __ldg(xp + off); });
  }
  if (interior) {
#pragma unroll
    for (int o = 0; o < NS; ++o) {
      const int ox = o % W - R, oy = (o / W) % W - R, oz = DIM == 3 ? o / (W * W) - R : 0;
      const i64 off = ox + sy * oy + sz * oz;
      // symmetric operator: a backward entry A(i, i+o) is read as A(i+o, i), the neighbour's
      // forward entry, so only the 14 forward / centre coefficient arrays are streamed
      const T a = o < NS / 2 ? __ldg(st + (NS - 1 - o) * m.nn + node + off) : __ldg(st + o * m.nn + node);
      s += a * __ldg(x + node + off);
    }
  } else {
#pragma unroll
    for (int o = 0; o < NS; ++o) {
      const int ox = o % W - R, oy = (o / W) % W - R, oz = DIM == 3 ? o / (W * W) - R : 0;
      const int jx = ix + ox, jy = iy + oy, jz = iz + oz;
      if (jx < 0 || jx >= m.nnx || jy < 0 || jy >= m.nny || jz < 0 || jz >= m.nnz) continue;
      const i64 off = ox + sy * oy + sz * oz;
      const T a = o < NS / 2 ? st[(NS - 1 - o) * m.nn + node + off] : st[o * m.nn + node];
      s += a * x[node + off];
    }
  }
  return s;
}

// The same sum over a vector given by a functor val(j) (j = node index within the block):
// for the fused Chebyshev kernels, whose input vector is formed on the fly.
template <int DIM, typename T, int R, typename V>
__device__ __forceinline__ T stencil_apply_f(const T* __restrict__ st, const DevMesh& m, i64 node, int ix, int iy,
                                             int iz, V val) {
  constexpr int NS = Sten<DIM, R>::V, W = Sten<DIM, R>::W;
  const i64 sy = m.nnx, sz = (i64)m.nnx * m.nny;
  T s = T(0);
  const bool interior = ix >= R && ix < m.nnx - R && iy >= R && iy < m.nny - R &&
                        (DIM == 2 || (iz >= R && iz < m.nnz - R));
  if (DIM == 3 && R == 1 && fast27(m, iy, iz, node, sy, sz))
    return stencil27_i32<T>(st, (int)m.nn, (int)node, (int)sy, (int)sz, [&](int off) { return val(node + off); });
  if (interior) {
#pragma unroll
    for (int o = 0; o < NS; ++o) {
      const int ox = o % W - R, oy = (o / W) % W - R, oz = DIM == 3 ? o / (W * W) - R : 0;
      const i64 off = ox + sy * oy + sz * oz;
      const T a = o < NS / 2 ? __ldg(st + (NS - 1 - o) * m.nn + node + off) : __ldg(st + o * m.nn + node);
      s += a * val(node + off);
    }
  } else {
#pragma unroll
    for (int o = 0; o < NS; ++o) {
      const int ox = o % W - R, oy = (o / W) % W - R, oz = DIM == 3 ? o / (W * W) - R : 0;
      const int jx = ix + ox, jy = iy + oy, jz = iz + oz;
      if (jx < 0 || jx >= m.nnx || jy < 0 || jy >= m.nny || jz < 0 || jz >= m.nnz) continue;
      const i64 off = ox + sy * oy + sz * oz;
      const T a = o < NS / 2 ? st[(NS - 1 - o) * m.nn + node + off] : st[o * m.nn + node];
      s += a * val(node + off);
    }
  }
  return s;
}

static dim3 block3(const DevMesh& m) { return m.dim == 3 ? dim3(32, 4, 2) : dim3(32, 8, 1); }
static dim3 grid3(const DevMesh& m) {
  const dim3 b = block3(m);
  return dim3((m.nnx + b.x - 1) / b.x, (m.nny + b.y - 1) / b.y, (m.nnz + b.z - 1) / b.z);
}
// smoother launches: one thread per node and block (node3b)
static dim3 grid3b(const DevMesh& m) {
  const dim3 g = grid3(m);
  return dim3(g.x, g.y, 2 * g.z);
}

// k_prolong: one thread per fine x-pair (coarse column), fine row and plane
static dim3 grid_prolong(const DevMesh& mf, const DevMesh& mc) {
  const dim3 b = block3(mf);
  return dim3((mc.nnx + b.x - 1) / b.x, (mf.nny + b.y - 1) / b.y, (mf.nnz + b.z - 1) / b.z);
}

static int grid_nodes(i64 n) {
  i64 g = (n + 255) / 256;
  if (g > 148 * 32) g = 148 * 32;
  return (int)(g < 1 ? 1 : g);
}

// Galerkin coarse stencil: A_c(I, J) = sum_{i,j} P(i,I) A(i,j) P(j,J). The fine stencil entry
// A(i, i+o2) with i = 2I + o1 reaches the coarse offsets J - I of the (one or two per axis)
// coarse nodes interpolating to 2I + o1 + o2. The offset o1 is a template parameter and the o2
// loop is unrolled, so every accumulator index is a compile-time constant and the 3^dim
// accumulators stay in registers.
template <int DIM, typename T, int RF, int O1>
__device__ __forceinline__ void rap_row(const DevMesh& mf, const T* __restrict__ stf, int cx, int cy, int cz,
                                        T* acc) {
  constexpr int NS = Sten<DIM, RF>::V, WF = Sten<DIM, RF>::W;
  constexpr int o1x = O1 % 3 - 1, o1y = (O1 / 3) % 3 - 1, o1z = DIM == 3 ? O1 / 9 - 1 : 0;
  const int fx = 2 * cx + o1x, fy = 2 * cy + o1y, fz = 2 * cz + o1z;
  if (fx < 0 || fx >= mf.nnx || fy < 0 || fy >= mf.nny || fz < 0 || fz >= mf.nnz) return;
  constexpr float w1f = (o1x ? 0.5f : 1.f) * (o1y ? 0.5f : 1.f) * (o1z ? 0.5f : 1.f);
  const T* sp = stf + fx + (i64)mf.nnx * (fy + (i64)mf.nny * fz);
#pragma unroll
  for (int o2 = 0; o2 < NS; ++o2) {
    const int o2x = o2 % WF - RF, o2y = (o2 / WF) % WF - RF, o2z = DIM == 3 ? o2 / (WF * WF) - RF : 0;
    const int rx = o1x + o2x, ry = o1y + o2y, rz = o1z + o2z;
    const T v = T(w1f) * __ldg(sp + (i64)o2 * mf.nn);
    // per axis: even r -> coarse offset r/2 (weight 1); odd r -> (r-1)/2 and (r+1)/2 (1/2 each)
#pragma unroll
    for (int c = 0; c < (1 << DIM); ++c) {
      const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
      if (((rx & 1) == 0 && bx) || ((ry & 1) == 0 && by) || (DIM == 3 && (rz & 1) == 0 && bz)) continue;
      const int jx = (rx & 1) ? (rx - 1) / 2 + bx : rx / 2;
      const int jy = (ry & 1) ? (ry - 1) / 2 + by : ry / 2;
      const int jz = DIM == 3 ? ((rz & 1) ? (rz - 1) / 2 + bz : rz / 2) : 0;
      // a radius-2 fine stencil (Q2 lattice) reaches coarse offsets up to 2 only through
      // entries that are structurally zero (nodes of different elements): skip them
      if (jx < -1 || jx > 1 || jy < -1 || jy > 1 || jz < -1 || jz > 1) continue;
      const T ww = ((rx & 1) ? T(0.5) : T(1)) * ((ry & 1) ? T(0.5) : T(1)) * (DIM == 3 && (rz & 1) ? T(0.5) : T(1));
      acc[(jx + 1) + 3 * (jy + 1) + (DIM == 3 ? 9 * (jz + 1) : 0)] += v * ww;
    }
  }
}

template <int DIM, typename T, int RF, int... O1>
__device__ __forceinline__ void rap_rows(const DevMesh& mf, const T* __restrict__ stf, int cx, int cy, int cz, T* acc,
                                         std::integer_sequence<int, O1...>) {
  (rap_row<DIM, T, RF, O1>(mf, stf, cx, cy, cz, acc), ...);
}

// fine stencils of radius RF (1, or 2 on the Q2 lattice), coarse stencils of radius 1
template <int DIM, typename T, int RF = 1>
__global__ void __launch_bounds__(256, 2) k_rap(DevMesh mf, DevMesh mc, const T* __restrict__ stf, T* __restrict__ stc) {
  constexpr int NS = Pow3<DIM>::V, NSF = Sten<DIM, RF>::V;
  int cx, cy, cz;
  i64 I;
  if (!node3(mc, cx, cy, cz, I)) return;
  for (int blk = 0; blk < 2; ++blk) {
    T acc[NS];
#pragma unroll
    for (int o = 0; o < NS; ++o) acc[o] = T(0);
    rap_rows<DIM, T, RF>(mf, stf + (i64)blk * NSF * mf.nn, cx, cy, cz, acc, std::make_integer_sequence<int, NS>{});
#pragma unroll
    for (int o = 0; o < NS; ++o) stc[((i64)blk * NS + o) * mc.nn + I] = acc[o];
  }
}

// D^-1 and the Gershgorin bound max_i sum_j |a_ij| / a_ii per block.
template <int DIM, typename T, int R = 1>
__global__ void k_gersh(DevMesh m, const T* __restrict__ st, T* __restrict__ dinv, double* __restrict__ partials) {
  constexpr int NS = Sten<DIM, R>::V;
  constexpr int C = NS / 2;
  __shared__ T red[2][256];
  T mx[2] = {T(0), T(0)};
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < m.nn; i += (i64)gridDim.x * blockDim.x) {
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      T s = T(0);
#pragma unroll
      for (int o = 0; o < NS; ++o) s += fabs(st[(blk * NS + o) * m.nn + i]);
      const T c = st[(blk * NS + C) * m.nn + i];
      const T ci = T(1) / c;
      dinv[blk * m.nn + i] = ci;
      mx[blk] = fmax(mx[blk], s * ci);
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
    partials[2 * blockIdx.x] = (double)red[0][0];
    partials[2 * blockIdx.x + 1] = (double)red[1][0];
  }
}

// out[b] = max over the nb per-block partial maxima (one block of 256 threads)
__global__ void k_max_partials(int nb, const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double red[2][256];
  double v0 = 0.0, v1 = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    v0 = fmax(v0, partials[2 * b]);
    v1 = fmax(v1, partials[2 * b + 1]);
  }
  red[0][threadIdx.x] = v0;
  red[1][threadIdx.x] = v1;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + w]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) out[threadIdx.x] = red[threadIdx.x][0];
}

// ---------------------------------------------------------------------------
// Chebyshev smoother, residual, transfers
// ---------------------------------------------------------------------------
// resident 256-thread blocks per SM the smoother kernels are compiled for
#ifndef TUSAS_SMOOTH_MINB
#define TUSAS_SMOOTH_MINB 8
#endif

// the 125-point kernels of the hex lattice get a larger register budget (4 blocks per SM)
template <int DIM, int R>
struct SmoothMinB {
  static const int V = (DIM == 3 && R == 2) ? 4 : TUSAS_SMOOTH_MINB;
};
// Coarse levels whose grid fits one wave at 2 blocks per SM take a variant compiled for 2
// blocks per SM (128 registers): there the launch is bound by the latency of each thread's 54
// stencil loads, which the larger budget keeps in flight at once instead of in several
// dependent rounds (7.2 instead of 8.7 us per launch on a 33 x 25 x 9 level; a 702-block
// level ran 2 us slower with it than with all its blocks resident at 32 registers).
// Grids of up to 3 blocks per SM (the 33 x 33 x 17 coarsest level of a 256 x 256 x 128 box: 324
// blocks) take a 3-blocks-per-SM variant (up to 85 registers): every block is resident either
// way, so the larger budget costs no occupancy.
static const int SMOOTH_LAT_MINB = 2, SMOOTH_LAT3_MINB = 3;
static int smooth_latency_grid(dim3 g) {
  const long long nb = (long long)g.x * g.y * g.z;
  return nb <= 148LL * SMOOTH_LAT_MINB ? SMOOTH_LAT_MINB : nb <= 148LL * SMOOTH_LAT3_MINB ? SMOOTH_LAT3_MINB : 0;
}

template <typename T>
struct Coef2 {
  T a[2], b[2];
};

// r = D^-1 (b - A x) (or D^-1 b if x == nullptr, and then x = 0); d = r * it
template <int DIM, typename T, int R = 1, int MB = SmoothMinB<DIM, R>::V>
__global__ void __launch_bounds__(256, MB) k_cheb_init(DevMesh m, const T* __restrict__ st, const T* __restrict__ dinv, const T* __restrict__ bvec,
                            T* __restrict__ x, int zero_x, T* __restrict__ r, T* __restrict__ d, Coef2<T> it) {
  constexpr int NS = Sten<DIM, R>::V;
  {
    int ix, iy, iz, blk;
    i64 i;
    if (!node3b(m, ix, iy, iz, i, blk)) return;
    T v = bvec[blk * m.nn + i];
    if (zero_x)
      x[blk * m.nn + i] = T(0);
    else
      v -= stencil_apply<DIM, T, R>(st + blk * NS * m.nn, x + blk * m.nn, m, i, ix, iy, iz);
    const T rr = dinv[blk * m.nn + i] * v;
    r[blk * m.nn + i] = rr;
    d[blk * m.nn + i] = rr * (blk ? it.a[1] : it.a[0]);
  }
}

// x += d; if !last: r -= D^-1 A d; dout = c1 d + c2 r
template <int DIM, typename T, int R = 1, int MB = SmoothMinB<DIM, R>::V>
__global__ void __launch_bounds__(256, MB) k_cheb_step(DevMesh m, const T* __restrict__ st, const T* __restrict__ dinv, T* __restrict__ x,
                            T* __restrict__ r, const T* __restrict__ d, T* __restrict__ dout, Coef2<T> c, int last) {
  constexpr int NS = Sten<DIM, R>::V;
  {
    int ix, iy, iz, blk;
    i64 i;
    if (!node3b(m, ix, iy, iz, i, blk)) return;
    const i64 k = blk * m.nn + i;
    const T dk = d[k];
    x[k] += dk;
    if (!last) {
      const T ad = stencil_apply<DIM, T, R>(st + blk * NS * m.nn, d + blk * m.nn, m, i, ix, iy, iz);
      const T rr = r[k] - dinv[k] * ad;
      r[k] = rr;
      dout[k] = (blk ? c.a[1] : c.a[0]) * dk + (blk ? c.b[1] : c.b[0]) * rr;
    }
  }
}

// The last Chebyshev step with a stencil product of the post-smoothing on the finest level,
// with the deferred step and the widening to FP64 folded in: z = x + d + dout, where
// x + d and dout = c1 d + c2 (r - D^-1 A d) are what k_cheb_step would store (the same
// rounding) and the final x += dout was left to the reader of x.
template <int DIM, typename T, int R = 1, int MB = SmoothMinB<DIM, R>::V>
__global__ void __launch_bounds__(256, MB) k_cheb_step_out(DevMesh m, const T* __restrict__ st, const T* __restrict__ dinv,
                                                           const T* __restrict__ x, const T* __restrict__ r,
                                                           const T* __restrict__ d, Coef2<T> c,
                                                           double* __restrict__ z) {
  constexpr int NS = Sten<DIM, R>::V;
  int ix, iy, iz, blk;
  i64 i;
  if (!node3b(m, ix, iy, iz, i, blk)) return;
  const i64 k = blk * m.nn + i;
  const T dk = d[k];
  const T xk = x[k] + dk;
  const T ad = stencil_apply<DIM, T, R>(st + blk * NS * m.nn, d + blk * m.nn, m, i, ix, iy, iz);
  const T rr = r[k] - dinv[k] * ad;
  const T dn = (blk ? c.a[1] : c.a[0]) * dk + (blk ? c.b[1] : c.b[0]) * rr;
  z[k] = (double)(xk + dn);
}

// The last Chebyshev step with a stencil product of a pre-smoothing, with the deferred step
// folded in: xout = (x + d) + dout, the sum k_resid_p would form at every neighbour (the same
// rounding), so the residual after the smoothing reads one array. Neither x, r nor dout is
// needed afterwards.
template <int DIM, typename T, int R = 1, int MB = SmoothMinB<DIM, R>::V>
__global__ void __launch_bounds__(256, MB) k_cheb_step_x(DevMesh m, const T* __restrict__ st, const T* __restrict__ dinv,
                                                         const T* __restrict__ x, const T* __restrict__ r,
                                                         const T* __restrict__ d, Coef2<T> c, T* __restrict__ xout) {
  constexpr int NS = Sten<DIM, R>::V;
  int ix, iy, iz, blk;
  i64 i;
  if (!node3b(m, ix, iy, iz, i, blk)) return;
  const i64 k = blk * m.nn + i;
  const T dk = d[k];
  const T xk = x[k] + dk;
  const T ad = stencil_apply<DIM, T, R>(st + blk * NS * m.nn, d + blk * m.nn, m, i, ix, iy, iz);
  const T rr = r[k] - dinv[k] * ad;
  const T dn = (blk ? c.a[1] : c.a[0]) * dk + (blk ? c.b[1] : c.b[0]) * rr;
  xout[k] = xk + dn;
}

template <int DIM, typename T, int R = 1, int MB = SmoothMinB<DIM, R>::V>
__global__ void __launch_bounds__(256, MB) k_resid(DevMesh m, const T* __restrict__ st, const T* __restrict__ bvec, const T* __restrict__ x,
                        T* __restrict__ res) {
  constexpr int NS = Sten<DIM, R>::V;
  {
    int ix, iy, iz, blk;
    i64 i;
    if (!node3b(m, ix, iy, iz, i, blk)) return;
    res[blk * m.nn + i] =
        bvec[blk * m.nn + i] - stencil_apply<DIM, T, R>(st + blk * NS * m.nn, x + blk * m.nn, m, i, ix, iy, iz);
  }
}

// Fused first Chebyshev step from x = 0 (the zero-x k_cheb_init followed by the first
// k_cheb_step, same arithmetic): r0 = D^-1 b, d0 = a0 r0, x = d0, r = r0 - D^-1 A d0,
// dout = c1 d0 + c2 r (requires degree >= 2, so the first step is not the last). db = D^-1 b,
// formed by the kernel that produced b (k_to_t, k_restrict), so the stencil reads one array at
// the 27 neighbours instead of two.
template <int DIM, typename T, int R = 1, int MB = SmoothMinB<DIM, R>::V>
__global__ void __launch_bounds__(256, MB)
    k_cheb_first(DevMesh m, const T* __restrict__ st, const T* __restrict__ dinv, const T* __restrict__ db,
                 T* __restrict__ x, T* __restrict__ r, T* __restrict__ dout, Coef2<T> it, Coef2<T> c) {
  constexpr int NS = Sten<DIM, R>::V;
  int ix, iy, iz, blk;
  i64 i;
  if (!node3b(m, ix, iy, iz, i, blk)) return;
  const i64 k = blk * m.nn + i;
  const T a0 = blk ? it.a[1] : it.a[0];
  const T* dbv = db + blk * m.nn;
  const T r0 = db[k];
  const T dk = r0 * a0;
  x[k] = dk;
  const T ad = stencil_apply_f<DIM, T, R>(st + blk * NS * m.nn, m, i, ix, iy, iz,
                                          [&](i64 j) { return __ldg(dbv + j) * a0; });
  const T rr = r0 - dinv[k] * ad;
  r[k] = rr;
  dout[k] = (blk ? c.a[1] : c.a[0]) * dk + (blk ? c.b[1] : c.b[0]) * rr;
}

// Residual with the last Chebyshev update folded in: x' = x + p (p the pending
// direction), res = b - A x', x' written to xout (a buffer other than x and p).
template <int DIM, typename T, int R = 1, int MB = SmoothMinB<DIM, R>::V>
__global__ void __launch_bounds__(256, MB)
    k_resid_p(DevMesh m, const T* __restrict__ st, const T* __restrict__ bvec, const T* __restrict__ x,
              const T* __restrict__ p, T* __restrict__ xout, T* __restrict__ res) {
  constexpr int NS = Sten<DIM, R>::V;
  int ix, iy, iz, blk;
  i64 i;
  if (!node3b(m, ix, iy, iz, i, blk)) return;
  const i64 k = blk * m.nn + i;
  const T* xv = x + blk * m.nn;
  const T* pv = p + blk * m.nn;
  xout[k] = x[k] + p[k];
  res[k] = bvec[k] - stencil_apply_f<DIM, T, R>(st + blk * NS * m.nn, m, i, ix, iy, iz,
                                                [&](i64 j) { return __ldg(xv + j) + __ldg(pv + j); });
}

// One smoother-type launch on level LV (both blocks): the kernel instance for the level's
// dimension and stencil radius, and for radius-1 levels that do not fill the GPU the
// latency variants (SMOOTH_LAT_MINB, SMOOTH_LAT3_MINB). T and st come from the caller.
#define TUSAS_SMOOTH_LAUNCH(KERN, LV, ...)                                                       \
  do {                                                                                          \
    const dim3 g_ = grid3b((LV).m), b_ = block3((LV).m);                                        \
    const int lat_ = smooth_latency_grid(g_);                                                   \
    if ((LV).m.dim == 3 && (LV).r == 2)                                                         \
      KERN<3, T, 2><<<g_, b_, 0, st>>>(__VA_ARGS__);                                            \
    else if ((LV).m.dim == 3 && lat_ == SMOOTH_LAT_MINB)                                        \
      KERN<3, T, 1, SMOOTH_LAT_MINB><<<g_, b_, 0, st>>>(__VA_ARGS__);                           \
    else if ((LV).m.dim == 3 && lat_ == SMOOTH_LAT3_MINB)                                       \
      KERN<3, T, 1, SMOOTH_LAT3_MINB><<<g_, b_, 0, st>>>(__VA_ARGS__);                          \
    else if ((LV).m.dim == 3)                                                                   \
      KERN<3, T><<<g_, b_, 0, st>>>(__VA_ARGS__);                                               \
    else if ((LV).r == 2)                                                                       \
      KERN<2, T, 2><<<g_, b_, 0, st>>>(__VA_ARGS__);                                            \
    else if (lat_ == SMOOTH_LAT_MINB)                                                           \
      KERN<2, T, 1, SMOOTH_LAT_MINB><<<g_, b_, 0, st>>>(__VA_ARGS__);                           \
    else if (lat_ == SMOOTH_LAT3_MINB)                                                          \
      KERN<2, T, 1, SMOOTH_LAT3_MINB><<<g_, b_, 0, st>>>(__VA_ARGS__);                          \
    else                                                                                        \
      KERN<2, T><<<g_, b_, 0, st>>>(__VA_ARGS__);                                               \
    count_launches(1);                                                                          \
  } while (0)

// b_c(I) = sum_i P(i, I) res(i) over the fine nodes within distance 1 of 2I (interior coarse
// nodes, whose 3^dim fine neighbours all exist, skip the bounds tests; same order of the sum),
// and if db_c is given D_c^-1 b_c there (for k_cheb_first on the coarse level)
template <int DIM, typename T>
__global__ void k_restrict(DevMesh mf, DevMesh mc, const T* __restrict__ res, T* __restrict__ bc,
                           const T* __restrict__ dinv_c, T* __restrict__ db_c) {
  constexpr int NS = Pow3<DIM>::V;
  {
    int cx, cy, cz;
    i64 I;
    if (!node3(mc, cx, cy, cz, I)) return;
    const bool interior = cx >= 1 && cx < mc.nnx - 1 && cy >= 1 && cy < mc.nny - 1 &&
                          (DIM == 2 || (cz >= 1 && cz < mc.nnz - 1));
    if (interior) {
      const i64 fsy = mf.nnx, fsz = (i64)mf.nnx * mf.nny;
      const i64 fc = 2 * (i64)cx + fsy * (2 * (i64)cy) + fsz * (2 * (i64)cz);
#pragma unroll
      for (int blk = 0; blk < 2; ++blk) {
        const T* r = res + blk * mf.nn + fc;
        T s = T(0);
#pragma unroll
        for (int o = 0; o < NS; ++o) {
          const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = DIM == 3 ? o / 9 - 1 : 0;
          const T w = (ox ? T(0.5) : T(1)) * (oy ? T(0.5) : T(1)) * (oz ? T(0.5) : T(1));
          s += w * r[ox + fsy * oy + fsz * oz];
        }
        bc[blk * mc.nn + I] = s;
        if (db_c) db_c[blk * mc.nn + I] = dinv_c[blk * mc.nn + I] * s;
      }
      return;
    }
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
      if (db_c) db_c[blk * mc.nn + I] = dinv_c[blk * mc.nn + I] * s;
    }
  }
}

// x_f(i) += sum_J P(i, J) (x_c(J) + p_c(J)); p_c: the coarse level's pending Chebyshev
// direction, or null. Fine node i = 2J + a (a_d in {0, 1}) interpolates between the coarse
// nodes J and J + a, axis by axis (x first) as the mean of the two values: where a_d = 0 both
// are the same node and the mean is exact, so every node takes the same branch-free path. One
// thread takes the fine x-pair 2j, 2j + 1 of one row in both blocks: the pair reads the same 2^dim
// coarse values (the last coarse column has no odd fine node). Grid: grid_prolong.
template <int DIM, typename T>
__global__ void k_prolong(DevMesh mf, DevMesh mc, const T* __restrict__ xc, const T* __restrict__ pc,
                          T* __restrict__ xf) {
  const int jx = blockIdx.x * blockDim.x + threadIdx.x;
  const int fy = blockIdx.y * blockDim.y + threadIdx.y;
  const int fz = blockIdx.z * blockDim.z + threadIdx.z;
  if (jx >= mc.nnx || fy >= mf.nny || fz >= mf.nnz) return;
  const i64 sy = mc.nnx, sz = (i64)mc.nnx * mc.nny;
  const i64 J0 = jx + sy * (fy >> 1) + sz * (fz >> 1);
  const bool odd = jx + 1 < mc.nnx;  // fine node 2 jx + 1 exists
  const i64 dx = odd ? 1 : 0, dy = (fy & 1) ? sy : 0, dz = (DIM == 3 && (fz & 1)) ? sz : 0;
  const i64 i = 2 * (i64)jx + (i64)mf.nnx * (fy + (i64)mf.nny * fz);
  const T half = T(0.5);
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    const T* xb = xc + blk * mc.nn;
    const T* pb = pc ? pc + blk * mc.nn : nullptr;
    auto cv = [&](i64 J) { return pb ? xb[J] + pb[J] : xb[J]; };
    // c[z][y][x]: the coarse values at J0 + (x ? dx : 0) + (y ? dy : 0) + (z ? dz : 0)
    T c[DIM == 3 ? 2 : 1][2][2];
#pragma unroll
    for (int z = 0; z < (DIM == 3 ? 2 : 1); ++z) {
      const i64 Jz = J0 + (z ? dz : 0);
      c[z][0][0] = cv(Jz);
      c[z][0][1] = cv(Jz + dx);
      c[z][1][0] = cv(Jz + dy);
      c[z][1][1] = cv(Jz + dy + dx);
    }
    // even node: both x values are the node itself (a_x = 0); odd node: the x-pair's two columns
    auto plane = [&](int z, int ox) {
      const T e0 = half * (c[z][0][0] + c[z][0][ox]);
      const T e1 = half * (c[z][1][0] + c[z][1][ox]);
      return half * (e0 + e1);
    };
    T ve = plane(0, 0), vo = plane(0, 1);
    if constexpr (DIM == 3) {
      ve = half * (ve + plane(1, 0));
      vo = half * (vo + plane(1, 1));
    }
    T* xo = xf + blk * mf.nn + i;
    xo[0] += ve;
    if (odd) xo[1] += vo;
  }
}

// b = r in the smoother precision, and if db is given D^-1 b (for k_cheb_first)
template <typename T>
__global__ void k_to_t(i64 n, const double* __restrict__ r, T* __restrict__ b, const T* __restrict__ dinv,
                       T* __restrict__ db) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const T bi = narrow<T>(r[i]);
    b[i] = bi;
    if (db) db[i] = dinv[i] * bi;
  }
}
// z = x (+ p, the pending Chebyshev direction, if not null), widened to FP64
template <typename T>
__global__ void k_from_t(i64 n, const T* __restrict__ x, const T* __restrict__ p, double* __restrict__ z) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    z[i] = (double)(p ? x[i] + p[i] : x[i]);
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
  if (m.order == 2 && kind == 1) {
    PrecondLevel L = {};
    L.m = m;
    L.nn = m.nn;
    cudaError_t e = dev_malloc(&L.dinv, esz * 2 * m.nn);
    if (e != cudaSuccess) return e;
    lv.push_back(L);  // destroy() frees what was allocated
    bytes += (esz + sizeof(double)) * 2 * m.nn;
    return dev_malloc(&diag, sizeof(double) * 2 * m.nn);
  }
  const int nlev = kind == 1 ? 1 : (levels < 1 ? 1 : levels);
  // Q2 (2D): the finest level is the node lattice of spacing h/2 with 25-point stencils; its
  // coarsening by 2 is the element-vertex grid (the Q1 space embedded in the Q2 space)
  DevMesh cur = m;
  if (m.order == 2) {
    cur.order = 1;
    cur.nx = 2 * m.nx;
    cur.ny = 2 * m.ny;
    if (m.dim == 3) cur.nz = 2 * m.nz;
    cur.ne = (i64)cur.nx * cur.ny * (m.dim == 3 ? cur.nz : 1);
    cur.h = 0.5 * m.h;
  }
  for (int l = 0; l < nlev; ++l) {
    PrecondLevel L = {};
    L.m = cur;
    L.nn = cur.nn;
    L.r = (l == 0 && m.order == 2) ? 2 : 1;
    const int NS = L.r == 2 ? (m.dim == 3 ? 125 : 25) : (m.dim == 3 ? 27 : 9);
    lv.push_back(L);  // allocated in place: destroy() frees a partly allocated level too
    PrecondLevel& Lb = lv.back();
    void** bufs[] = {&Lb.dinv, &Lb.b, &Lb.x, &Lb.r_, &Lb.d, &Lb.d2, &Lb.res};
    cudaError_t e = dev_malloc(&Lb.st, esz * 2 * NS * cur.nn);
    if (e != cudaSuccess) return e;
    bytes += esz * 2 * NS * cur.nn;
    const int nvec = kind == 1 ? 1 : 7;
    for (int v = 0; v < nvec; ++v) {
      e = dev_malloc(bufs[v], esz * 2 * cur.nn);
      if (e != cudaSuccess) return e;
      bytes += esz * 2 * cur.nn;
    }
    if (!can_coarsen(cur)) break;
    cur = coarsen(cur);
  }
  cudaError_t e = dev_malloc(&gersh_partials, sizeof(double) * 2 * 148 * 32);
  if (e != cudaSuccess) return e;
  return dev_malloc(&lmax_dev, sizeof(double) * 2 * lv.size());
}

void Precond::destroy() {
  for (auto& L : lv) {
    void* bufs[] = {L.st, L.dinv, L.b, L.x, L.r_, L.d, L.d2, L.res};
    for (void* p : bufs)
      if (p) dev_free(p);
  }
  lv.clear();
  dev_free(gersh_partials);
  dev_free(lmax_dev);
  dev_free(diag);
  gersh_partials = lmax_dev = diag = nullptr;
}

template <typename T>
cudaError_t Precond::setup_t(const ElemCtx& c, double theta, const double* U, const double* Un, cudaStream_t st) {
  const DevMesh& m = c.m;
  PrecondLevel& L0 = lv[0];
  if (m.order == 2 && kind == 1) {
    // point Jacobi: element pass for diag(M11), diag(M22), then the reciprocals
    cudaError_t e = elem_run(M_DIAG, c, U, Un, nullptr, diag, nullptr, st);
    if (e != cudaSuccess) return e;
    k_recip<T><<<grid_nodes(2 * m.nn), 256, 0, st>>>(2 * m.nn, diag, (T*)L0.dinv);
    count_launches(1);
    return cudaGetLastError();
  }
  if (m.order == 2) {
    // multigrid: 25- or 125-point stencils on the Q2 node lattice, then the Galerkin levels
    // below (for hexes the vertex level comes from the same fill)
    cudaError_t e = m.dim == 3 ? q2h_stencil_fill<T>(c, U, Un, (T*)L0.st, lv.size() > 1 ? (T*)lv[1].st : nullptr, st)
                               : q2_stencil_fill<T>(c, U, Un, (T*)L0.st, st);
    if (e != cudaSuccess) return e;
    return galerkin_and_bounds<T>(st);
  }
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
  const double wg = m.dim == 3 ? pow(m.h / 2, 3) : pow(m.h / 2, 2);
  A.w = (T)wg;
  A.ih2 = (T)(1.0 / (m.h * m.h));
  const DevPhys& P = c.P;
  A.guard = (T)TUSAS_GUARD_Q;
  A.one_m3e = (T)(1.0 - 3.0 * P.eps4);
  A.four_e = (T)(4.0 * P.eps4);
  A.omk = (T)(1.0 - P.k);
  A.half_opk = (T)(0.5 * (1.0 + P.k));
  A.half_omk = (T)(0.5 * (1.0 - P.k));
  A.wm1 = (T)(wg * P.tau0 * P.idt);
  A.wk1 = (T)(wg * theta * P.W0 * P.W0);
  A.wm2 = (T)(wg * P.idt);
  A.wk2 = (T)(wg * theta * P.D);
  A.U = U;
  A.Un = Un;
  A.st = (T*)L0.st;
  cudaError_t e = cudaSuccess;
  if (m.dim == 3) {
    using FT = FillTile<3, T>;
    const size_t smem = sizeof(T) * 2 * 27 * FT::NEL;
    const dim3 grid(ceil_div(m.nnx, FT::X), ceil_div(m.nny, FT::Y), ceil_div(m.nnz, FT::Z));
    if (c.P.model == 0) {
      e = cudaFuncSetAttribute(k_stencil_fill<3, 0, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_stencil_fill<3, 0, T><<<grid, FT::THREADS, smem, st>>>(A);
    } else {
      e = cudaFuncSetAttribute(k_stencil_fill<3, 1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_stencil_fill<3, 1, T><<<grid, FT::THREADS, smem, st>>>(A);
    }
    count_launches(1);
  } else {
    using FT = FillTile<2, T>;
    const size_t smem = sizeof(T) * 2 * 9 * FT::NEL;
    const dim3 grid(ceil_div(m.nnx, FT::X), ceil_div(m.nny, FT::Y), 1);
    if (c.P.model == 0)
      k_stencil_fill<2, 0, T><<<grid, FT::THREADS, smem, st>>>(A);
    else
      k_stencil_fill<2, 1, T><<<grid, FT::THREADS, smem, st>>>(A);
    count_launches(1);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return galerkin_and_bounds<T>(st);
}

// Galerkin coarse stencils of levels 1.., D^-1 and the Gershgorin bounds of every level.
// Synchronises once (the bounds are host scalars of the Chebyshev smoother).
template <typename T>
cudaError_t Precond::galerkin_and_bounds(cudaStream_t st) {
  const int dim = lv[0].m.dim;
  for (size_t l = 1; l < lv.size(); ++l) {
    const PrecondLevel& F = lv[l - 1];
    const PrecondLevel& C = lv[l];
    if (dim == 3 && F.r == 2) continue;  // the hex vertex level is filled with the lattice level
    if (dim == 3)
      k_rap<3, T><<<grid3(C.m), block3(C.m), 0, st>>>(F.m, C.m, (const T*)F.st, (T*)C.st);
    else if (F.r == 2)
      k_rap<2, T, 2><<<grid3(C.m), block3(C.m), 0, st>>>(F.m, C.m, (const T*)F.st, (T*)C.st);
    else
      k_rap<2, T><<<grid3(C.m), block3(C.m), 0, st>>>(F.m, C.m, (const T*)F.st, (T*)C.st);
    count_launches(1);
  }
  for (size_t l = 0; l < lv.size(); ++l) {
    const int nb = grid_nodes(lv[l].nn);
    if (dim == 3 && lv[l].r == 2)
      k_gersh<3, T, 2><<<nb, 256, 0, st>>>(lv[l].m, (const T*)lv[l].st, (T*)lv[l].dinv, gersh_partials);
    else if (dim == 3)
      k_gersh<3, T><<<nb, 256, 0, st>>>(lv[l].m, (const T*)lv[l].st, (T*)lv[l].dinv, gersh_partials);
    else if (lv[l].r == 2)
      k_gersh<2, T, 2><<<nb, 256, 0, st>>>(lv[l].m, (const T*)lv[l].st, (T*)lv[l].dinv, gersh_partials);
    else
      k_gersh<2, T><<<nb, 256, 0, st>>>(lv[l].m, (const T*)lv[l].st, (T*)lv[l].dinv, gersh_partials);
    count_launches(1);
    k_max_partials<<<1, 256, 0, st>>>(nb, gersh_partials, lmax_dev + 2 * l);
    count_launches(1);
  }
  cudaError_t e = cudaGetLastError();
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
cudaError_t Precond::cheb(int l, bool zero_x, int degree, cudaStream_t st, double* zout, bool* zdone, bool fold) {
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
  auto next_coef = [&]() {
    for (int b = 0; b < 2; ++b) {
      const double rn = 1.0 / (2.0 * sigma[b] - rho[b]);
      cc.a[b] = (T)(rn * rho[b]);
      cc.b[b] = (T)(2.0 * rn / delta[b]);
      rho[b] = rn;
    }
  };
  const T *S = (const T*)L.st, *Di = (const T*)L.dinv, *B = (const T*)L.b;
  T *X = (T*)L.x, *Rr = (T*)L.r_;
  T* dcur = (T*)L.d;
  T* dnext = (T*)L.d2;
  L.pend = nullptr;
  // FP32: fused first step and deferred last step; the FP64 variants of the fused kernels
  // spill at the 32-register budget of the smoother kernels and ran 40 % slower
  constexpr bool fuse = sizeof(T) == sizeof(float);
  int k0 = 0;
  if (fuse && zero_x && degree >= 2) {  // zero start: initialisation and first step in one pass
    next_coef();
    TUSAS_SMOOTH_LAUNCH(k_cheb_first, L, L.m, S, Di, (const T*)L.res, X, Rr, dnext, it, cc);  // res holds D^-1 b
    std::swap(dcur, dnext);
    k0 = 1;
  } else {
    TUSAS_SMOOTH_LAUNCH(k_cheb_init, L, L.m, S, Di, B, X, zero_x, Rr, dcur, it);
  }
  for (int kk = k0; kk < degree; ++kk) {
    const int last = kk == degree - 1;
    if (fuse && last) {  // the last step is x += d only: left to the next reader of x
      L.pend = dcur;
      break;
    }
    next_coef();
    if (fuse && zout && kk == degree - 2) {  // the result goes straight to z (FP64)
      TUSAS_SMOOTH_LAUNCH(k_cheb_step_out, L, L.m, S, Di, X, Rr, dcur, cc, zout);
      *zdone = true;
      L.pend = nullptr;
      return cudaGetLastError();
    }
    if (fuse && fold && kk == degree - 2) {  // the smoothed x, last step included, into the free buffer
      TUSAS_SMOOTH_LAUNCH(k_cheb_step_x, L, L.m, S, Di, X, Rr, dcur, cc, dnext);
      void* old_x = L.x;
      L.x = dnext;
      L.d = dcur;
      L.d2 = old_x;
      L.pend = nullptr;
      return cudaGetLastError();
    }
    TUSAS_SMOOTH_LAUNCH(k_cheb_step, L, L.m, S, Di, X, Rr, dcur, dnext, cc, last);
    std::swap(dcur, dnext);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t Precond::vcycle(int l, cudaStream_t st, double* zout, bool* zdone) {
  const int last = (int)lv.size() - 1;
  // below the finest level the smoothed x is read only by the prolongation: its last
  // stencil step writes x with the step's own direction added (fold), so the prolongation
  // reads one coarse array
  if (l == last) return cheb<T>(l, true, coarse_degree, st, nullptr, nullptr, true);
  cudaError_t e = cheb<T>(l, true, cheb_degree, st, nullptr, nullptr, true);
  if (e != cudaSuccess) return e;
  PrecondLevel& F = lv[l];
  PrecondLevel& C = lv[l + 1];
  const bool d3 = F.m.dim == 3;
  const T *S = (const T*)F.st, *B = (const T*)F.b;
  if (F.pend) {  // residual of x + pending direction; the updated x goes to the free direction buffer
    void** xo = F.pend == F.d ? &F.d2 : &F.d;
    const T *X = (const T*)F.x, *P = (const T*)F.pend;
    TUSAS_SMOOTH_LAUNCH(k_resid_p, F, F.m, S, B, X, P, (T*)*xo, (T*)F.res);
    std::swap(F.x, *xo);
    F.pend = nullptr;
  } else {
    TUSAS_SMOOTH_LAUNCH(k_resid, F, F.m, S, B, (const T*)F.x, (T*)F.res);
  }
  // FP32: D_c^-1 b_c into the coarse level's residual buffer for its k_cheb_first
  T* dbc = sizeof(T) == sizeof(float) ? (T*)C.res : nullptr;
  if (d3)
    k_restrict<3, T><<<grid3(C.m), block3(C.m), 0, st>>>(F.m, C.m, (const T*)F.res, (T*)C.b, (const T*)C.dinv, dbc);
  else
    k_restrict<2, T><<<grid3(C.m), block3(C.m), 0, st>>>(F.m, C.m, (const T*)F.res, (T*)C.b, (const T*)C.dinv, dbc);
  count_launches(1);
  e = vcycle<T>(l + 1, st);
  if (e != cudaSuccess) return e;
  if (d3)
    k_prolong<3, T><<<grid_prolong(F.m, C.m), block3(F.m), 0, st>>>(F.m, C.m, (const T*)C.x, (const T*)C.pend,
                                                                     (T*)F.x);
  else
    k_prolong<2, T><<<grid_prolong(F.m, C.m), block3(F.m), 0, st>>>(F.m, C.m, (const T*)C.x, (const T*)C.pend,
                                                                     (T*)F.x);
  count_launches(1);
  C.pend = nullptr;
  return cheb<T>(l, false, cheb_degree, st, zout, zdone, l > 0);
}

template <typename T>
cudaError_t Precond::apply_t(const double* r, double* z, cudaStream_t st, bool input_ready) {
  PrecondLevel& L0 = lv[0];
  const i64 n = 2 * L0.nn;
  if (kind == 1) {
    {
      k_jacobi<T><<<grid_nodes(n), 256, 0, st>>>(n, (const T*)L0.dinv, r, z);
      count_launches(1);
    }
    return cudaGetLastError();
  }
  if (!input_ready) {
    // FP32: D^-1 b into the level's residual buffer (free until its residual pass) for k_cheb_first
    T* db = sizeof(T) == sizeof(float) ? (T*)L0.res : nullptr;
    k_to_t<T><<<grid_nodes(n), 256, 0, st>>>(n, r, (T*)L0.b, (const T*)L0.dinv, db);
    count_launches(1);
  }
  bool zdone = false;
  cudaError_t e = vcycle<T>(0, st, z, &zdone);
  if (e != cudaSuccess) return e;
  if (!zdone) {
    k_from_t<T><<<grid_nodes(n), 256, 0, st>>>(n, (const T*)L0.x, (const T*)L0.pend, z);
    count_launches(1);
  }
  L0.pend = nullptr;
  return cudaGetLastError();
}

cudaError_t Precond::apply(const double* r, double* z, cudaStream_t st, bool input_ready) {
  if (kind == 0 || lv.empty()) return cudaErrorInvalidValue;  // identity is applied by the caller
  if (input_ready && !fp32_input(nullptr, nullptr, nullptr)) return cudaErrorInvalidValue;
  return fp32 ? apply_t<float>(r, z, st, input_ready) : apply_t<double>(r, z, st, false);
}

bool Precond::fp32_input(float** b, float** db, const float** dinv) const {
  if (kind != 2 || !fp32 || lv.empty()) return false;
  if (b) *b = (float*)lv[0].b;
  if (db) *db = (float*)lv[0].res;  // free until the level's residual pass (k_cheb_first reads it)
  if (dinv) *dinv = (const float*)lv[0].dinv;
  return true;
}

}  // namespace tusas
