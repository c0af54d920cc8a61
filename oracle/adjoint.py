"""Discrete adjoint of N backward-Euler steps for a linear functional S = w^T U_N.

Not in the paper (its Jacobian-free Newton-Krylov solver, Sec. 2.2, needs only
F and J v); this is the plain definition of the gradient of the discrete
solution map. With F_n(U_n, U_{n-1}; p) = 0 for n = 1..N:

  J_N^T lam_N = w,   J_n^T lam_n = -(dF_{n+1}/dU_n)^T lam_{n+1}  (n < N),
  dS/dp   = -sum_n lam_n^T dF_n/dp,
  dS/dU_0 = -(dF_1/dU_0)^T lam_1,

with J_n = dF_n/dU_n. Every Jacobian comes from ``jacobian`` (complex step);
the linear solves are sparse LU. The solid fraction S = int (1 + phi)/2 is
w^T U with w = half the consistent-mass row sums on the phi nodes (the exact
integral of the Q1 interpolant) plus the constant |Omega|/2.

Parity: pinned against central differences of the forward solve
(tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem, jacobian
from .solver import newton_direct


def solid_fraction_weights(mesh):
    """(w, c): S = w^T U + c equals int (1 + phi_h)/2 over the box.

    The integral of each nodal basis function is a product of 1D integrals:
    per element [h/2, h/2] for Q1 (trapezoid), [h/6, 2h/3, h/6] for Q2
    (Simpson), summed over the elements that share a node.
    """
    p = fem.order(mesh)
    elem_w = [0.5, 0.5] if p == 1 else [1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0]
    one_d = []
    for ne in fem.n_elems_axis(mesh):
        m = np.zeros(p * ne + 1)
        for e in range(ne):
            for a, wa in enumerate(elem_w):
                m[p * e + a] += wa * mesh.h
        one_d.append(m)
    mrow = one_d[0]
    for m in one_d[1:]:
        mrow = np.kron(m, mrow)  # x fastest
    w = np.concatenate([0.5 * mrow, np.zeros(mesh.n_nodes)])
    vol = np.prod([mesh.h * ne for ne in fem.n_elems_axis(mesh)])
    return w, 0.5 * vol


def forward(mesh, prm, U0, t0, dt, nsteps, rtol=1e-13):
    states = [U0.copy()]
    t = t0
    for _ in range(nsteps):
        U, ratio = newton_direct(mesh, prm, states[-1], t, dt, rtol=rtol)
        states.append(U)
        t += dt
    return states


def gradient(mesh, prm, states, t0, dt, w):
    """(dS/d eps4, dS/dU_0) for S = w^T U_N along the recorded states."""
    N = len(states) - 1
    lam_next = None
    g_eps = 0.0
    for n in range(N, 0, -1):
        t_prev = t0 + (n - 1) * dt
        rhs = w.copy() if n == N else np.zeros_like(w)
        if n < N:
            rhs -= jacobian.dF_dUn_T(mesh, prm, states[n + 1], states[n], t0 + n * dt, dt, lam_next)
        J = jacobian.sparse_jacobian(mesh, prm, states[n], states[n - 1], t_prev, dt)
        lam = spla.spsolve(J.T.tocsc(), rhs)
        g_eps -= lam @ jacobian.dF_deps4(mesh, prm, states[n], states[n - 1], t_prev, dt)
        lam_next = lam
    g0 = -jacobian.dF_dUn_T(mesh, prm, states[1], states[0], t0, dt, lam_next)
    return g_eps, g0
