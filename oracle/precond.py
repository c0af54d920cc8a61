"""Physics-based block-diagonal preconditioner M = diag(M11, M22) (Sec. 2.3.2, Eq. pre).

Blocks, the linearised forms of Eqs. (pref2) and (preconc2) in Karma-Rappel
units, evaluated pointwise at the Gauss points of the current Newton iterate:

  (M11)_ij = (1/dt) (tau0 B(u) a(p)^2 psi_j, psi_i) + theta (W0^2 a(p)^2 grad psi_j, grad psi_i)
  (M22)_ij = (1/dt) (A(phi^n) psi_j, psi_i)         + theta (D q(phi) grad psi_j, grad psi_i)

(the nodal index on a(theta_j) in Eqs. (m11)/(pref2) is read as a Gauss-point
evaluation; beta*Gamma of Eq. (m11) is 1 in these units; A(phi^n) replaces the
printed (1+k)/2 consistently with the residual). Both blocks are SPD.

Inversion (the paper uses algebraic multigrid with Gauss-Seidel or Chebyshev
smoothing, Sec. 4.1 and 4.4; this build uses the geometric equivalent on the
structured box):

* point Jacobi z = r / diag(M);
* geometric multigrid V-cycle per block: vertex-centred coarsening by 2 with
  (bi/tri)linear prolongation P, Galerkin coarse operators P^T A P,
  Chebyshev smoothing of the Jacobi-scaled operator (Saad, Iterative Methods
  for Sparse Linear Systems, Alg. 12.1) of degree ``cheb_degree`` before and
  after the coarse correction, degree ``coarse_degree`` on the coarsest level;
  eigenvalue interval [lmax/30, lmax] with lmax the Gershgorin bound
  max_i sum_j |a_ij| / a_ii of D^-1 A (a guaranteed upper bound, so the
  smoother never amplifies the highest modes; ten power iterations
  underestimated lmax of the M11 block by 12 % and made the cycle diverge).

Parity: assembly pinned by the textbook Q1 stencils; V-cycle pinned by its
convergence as a stationary iteration and by exactness on one level with an
exact coarse solve (tests/test_oracle_precond.py).
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np
import scipy.sparse as sp

from . import fem
from .residual import anisotropy, gather


def gp_coefficients(mesh, prm, U, Un, dt):
    """Per element and Gauss point: (cm11, ck11, cm22, ck22), shape (4, E, 2^dim)."""
    dim, h = mesh.dim, mesh.h
    elems = fem.all_elements(mesh)
    conn = fem.connectivity(mesh, elems)
    phi_e, u_e = gather(mesh, U, conn)
    phin_e, _ = gather(mesh, Un, conn)
    E = conn.shape[0]
    out = np.zeros((4, E, len(fem.gauss_rule(dim, fem.order(mesh)))))
    k = prm.k
    for gi, (xi, _) in enumerate(fem.gauss_rule(dim, fem.order(mesh))):
        N, G = fem.basis(dim, xi, h, fem.order(mesh))
        phi = phi_e @ N
        u = u_e @ N
        phin = phin_e @ N
        p = [phi_e @ G[d] for d in range(dim)]
        a, _, _, _ = anisotropy(prm, p)
        B = 1.0 + (1.0 - k) * u
        A = ((1.0 + k) - (1.0 - k) * phin) / 2.0
        mob = (1.0 - phi) / 2.0 if prm.model == 1 else np.ones_like(phi)
        out[0, :, gi] = prm.tau0 * B * a * a / dt
        out[1, :, gi] = prm.theta * prm.W0 ** 2 * a * a
        out[2, :, gi] = A / dt
        out[3, :, gi] = prm.theta * prm.D * mob
    return out, conn


def assemble(mesh, cm, ck, conn):
    """sum_e sum_g w (cm N N^T + ck G^T G) as a CSR matrix (N_nodes square)."""
    dim, h = mesh.dim, mesh.h
    n = mesh.n_nodes
    nl = conn.shape[1]
    E = conn.shape[0]
    Ke = np.zeros((E, nl, nl))
    for gi, (xi, wref) in enumerate(fem.gauss_rule(dim, fem.order(mesh))):
        N, G = fem.basis(dim, xi, h, fem.order(mesh))
        w = wref * h ** dim
        Ke += w * (cm[:, gi, None, None] * np.outer(N, N)[None] + ck[:, gi, None, None] * (G.T @ G)[None])
    rows = np.repeat(conn[:, :, None], nl, axis=2)
    cols = np.repeat(conn[:, None, :], nl, axis=1)
    return sp.coo_matrix((Ke.reshape(-1), (rows.reshape(-1), cols.reshape(-1))), shape=(n, n)).tocsr()


def blocks(mesh, prm, U, Un, dt):
    c, conn = gp_coefficients(mesh, prm, U, Un, dt)
    return assemble(mesh, c[0], c[1], conn), assemble(mesh, c[2], c[3], conn)


# ----------------------------------------------------------------------------
# geometric multigrid
# ----------------------------------------------------------------------------

def coarse_mesh(mesh):
    return dataclasses.replace(mesh, nx=mesh.nx // 2, ny=mesh.ny // 2,
                               nz=mesh.nz // 2 if mesh.dim == 3 else 0, h=2 * mesh.h)


def can_coarsen(mesh):
    return fem.order(mesh) == 1 and all(n % 2 == 0 and n >= 2 for n in fem.n_elems_axis(mesh))


def prolongation(mesh):
    """Vertex-centred (bi/tri)linear interpolation from the coarse to the fine nodes."""
    nnf = fem.n_nodes_axis(mesh)
    cm = coarse_mesh(mesh)
    grids = np.meshgrid(*[np.arange(n) for n in nnf], indexing="ij")
    fine_idx = [g.transpose().reshape(-1) for g in grids]
    fine_flat = fem.node_index(mesh, fine_idx)
    rows, cols, vals = [], [], []
    # per axis: even fine index 2I -> coarse I (weight 1); odd 2I+1 -> I and I+1 (1/2 each)
    for choice in itertools.product([0, 1], repeat=mesh.dim):
        ci = []
        w = np.ones(len(fine_flat))
        for d in range(mesh.dim):
            f = fine_idx[d]
            odd = f % 2 == 1
            if choice[d] == 0:
                ci.append(f // 2)
                w = w * np.where(odd, 0.5, 1.0)
            else:
                ci.append(f // 2 + 1)
                w = w * np.where(odd, 0.5, 0.0)
        ok = w != 0
        rows.append(fine_flat[ok])
        cols.append(fem.node_index(cm, [c[ok] for c in ci]))
        vals.append(w[ok])
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.n_nodes, cm.n_nodes))
    return P.tocsr()


def gershgorin(A):
    """Upper bound of the spectrum of D^-1 A: max over rows of sum_j |a_ij| / a_ii."""
    d = A.diagonal()
    return float((abs(A).sum(axis=1).A1 / d).max())


def chebyshev(A, dinv, b, x, lmin, lmax, degree):
    """Chebyshev iteration on D^-1 A x = D^-1 b, eigenvalues in [lmin, lmax] (Saad Alg. 12.1).

    ``x`` None means a zero initial guess (no matrix product for the first residual).
    """
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x is None:
        r = dinv * b
        x = np.zeros_like(b)
    else:
        r = dinv * (b - A @ x)
        x = x.copy()
    d = r / theta
    for kk in range(degree):
        x = x + d
        if kk == degree - 1:
            break
        r = r - dinv * (A @ d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x


class Hierarchy:
    """Galerkin hierarchy of one SPD block on the structured box."""

    def __init__(self, mesh, A, levels, cheb_degree=2, coarse_degree=10):
        self.A = [A]
        self.P = []
        self.meshes = [mesh]
        m = mesh
        while len(self.A) < levels and can_coarsen(m):
            P = prolongation(m)
            self.P.append(P)
            self.A.append((P.T @ self.A[-1] @ P).tocsr())
            m = coarse_mesh(m)
            self.meshes.append(m)
        self.dinv = [1.0 / Al.diagonal() for Al in self.A]
        self.lmax = [gershgorin(Al) for Al in self.A]
        self.cheb_degree = cheb_degree
        self.coarse_degree = coarse_degree

    def vcycle(self, b, level=0):
        A, dinv, lm = self.A[level], self.dinv[level], self.lmax[level]
        lo, hi = lm / 30.0, lm
        if level == len(self.A) - 1:
            return chebyshev(A, dinv, b, None, lo, hi, self.coarse_degree)
        x = chebyshev(A, dinv, b, None, lo, hi, self.cheb_degree)
        r = b - A @ x
        xc = self.vcycle(self.P[level].T @ r, level + 1)
        x = x + self.P[level] @ xc
        return chebyshev(A, dinv, b, x, lo, hi, self.cheb_degree)


def q2_lattice(mesh):
    """The Q2 node grid seen as a Q1 box of spacing h/2 (the multigrid hierarchy of a Q2 block).

    Its first coarsening by 2 is the grid of the Q2 element vertices, and the
    (bi)linear prolongation between the two is the exact embedding of the Q1
    space of the elements in their Q2 space, so the Galerkin product P^T A P of
    the assembled Q2 block is the Q1 operator with the Q2 quadrature
    (9-point, 27-point for hexes); the levels below are the Q1 hierarchy.
    """
    return dataclasses.replace(mesh, nx=2 * mesh.nx, ny=2 * mesh.ny, nz=2 * mesh.nz if mesh.dim == 3 else 0,
                               h=mesh.h / 2, order=1)


class Preconditioner:
    """z = M^-1 r for kind 0 (identity), 1 (point Jacobi), 2 (block Jacobi + GMG)."""

    def __init__(self, mesh, prm, U, Un, dt):
        self.kind = prm.precond
        self.n = mesh.n_nodes
        if self.kind == 0:
            return
        self.M11, self.M22 = blocks(mesh, prm, U, Un, dt)
        if self.kind == 1:
            self.d = np.concatenate([self.M11.diagonal(), self.M22.diagonal()])
        else:
            hm = q2_lattice(mesh) if fem.order(mesh) == 2 else mesh
            self.h11 = Hierarchy(hm, self.M11, prm.mg_levels, prm.cheb_degree, prm.coarse_degree)
            self.h22 = Hierarchy(hm, self.M22, prm.mg_levels, prm.cheb_degree, prm.coarse_degree)

    def apply(self, r):
        if self.kind == 0:
            return r.copy()
        if self.kind == 1:
            return r / self.d
        n = self.n
        return np.concatenate([self.h11.vcycle(r[:n]), self.h22.vcycle(r[n:])])
