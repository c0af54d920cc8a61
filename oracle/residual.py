"""Discrete residual F(U) of the coupled phase-field / solute (or temperature) system.

Follows Sec. 4.2, Eqs. (pf2), (lambda), (directional), (conc2), (jat), with the
four-fold anisotropy of Eq. (gs) and the theta-method of Eqs. (dpf)/(dc)/(theta)
(theta = 1 backward Euler, 1/2 Crank-Nicolson), in Karma-Rappel units
W0 = tau0 = 1 (Sec. 4.2, the nondimensionalisation paragraph). The pure metal is the same system with k = 1,
mobility q = 1, no antitrapping current and no frozen gradient (Karma-Rappel
phi + dimensionless temperature u).

Pointwise integrands at a Gauss point, with p = grad phi, g = grad u,
phihat = (phi - phi^n)/dt, B(u) = 1 + (1-k) u:

  a(p)   = 1 - 3 eps4 + 4 eps4 sum p_i^4 / |p|^4                          Eq. (gs)
  f_phi  = d/dp [ W0^2 |p|^2 a(p)^2 / 2 ]
         = W0^2 ( a^2 p + |p|^2 a da/dp )
  s_phi  = tau0 B(u) a^2 phihat - ( phi - phi^3 - lam (1-phi^2)^2 (u + G4) )
  s_u    = A(phi^n) (u - u^n)/dt - phihat B(u) / 2,  A = ((1+k) - (1-k) phi)/2
  f_u    = D q(phi) g + j,  q = (1-phi)/2 (alloy) or 1 (pure metal),
           j = W0 B(u) phihat p/|p| / (2 sqrt 2)  (alloy only)

and R_{phi,i} = sum_e sum_g w (s_phi psi_i + f_phi . grad psi_i), likewise R_u.

theta-method (Eqs. dpf, dc, theta): the time terms are evaluated as above
with (phi^{n+1} - phi^n)/dt; the bulk term and the fluxes D q(phi) grad u and
f_phi are weighted theta at level n+1 plus (1 - theta) at level n (G4 at the
level's own time). phihat in the antitrapping current and in the solute
source: ``phihat_form`` 1 (default), (phi^{n+1} - phi^n)/dt; ``phihat_form`` 0,
the estimate printed as Eq. (theta),
  phihat = theta (phi^{n+1} - phi^n)/dt + (1 - theta)(phi^n - phi^{n-1})/dt,
with phi^{n-1} = phi^n when no earlier level exists. Eq. (theta)'s estimate is
centred at t^n, so with it theta = 1/2 is only first order in time (pinned),
while Sec. 4.1.2 reports second order for Crank-Nicolson; form 1 gives second
order. The antitrapping current and the source take u, grad phi at n+1, as
printed in Eq. (conc2).
Readings of garbled or ambiguous passages (switchable where marked):

* anisotropic flux: the variational derivative of the gradient energy with
  sigma = a(p) (the printed forms of the extra anisotropy term are not
  dimensionally consistent);
* bulk term: phi - phi^3 - lam (1-phi^2)^2 (u + G4) (the printed G3(phi)(u+G4)
  would multiply phi - phi^3 by u and has no stationary flat front);
* time term ``time_form`` 0: tau0 B(u^{n+1}) a(p^{n+1})^2 (phi^{n+1}-phi^n)/dt;
  ``time_form`` 1: the printed difference of products
  tau0 ([B a^2 phi]^{n+1} - [B a^2 phi]^n)/dt;
* solute time coefficient A(phi^n) (the printed (1+k)/2 has no conserved
  quantity; with A at phi^n and B at u^{n+1} the sum over i of R_u is an exact
  difference quotient of the integral of A(phi)B(u)/(1-k), so solute is
  conserved to Newton tolerance);
* antitrapping ``jat_normalised`` 1: unit normal p/|p| (guarded), 0: p as printed;
* guard: where |p|^2 < 1e-20 the anisotropy is switched off (a = 1,
  f_phi = W0^2 p) and j = 0;
* frozen gradient G4 = (x_last - zT - Vp t^{n+1})/lT along the last axis
  (alloy with lT != 0), else 0; zT is the position of the reference isotherm
  at t = 0.

Parity: pinned (textbook Q1 stencils, flat interface, MMS second order,
conservation, symmetry; tests/test_oracle_residual.py).
"""
from __future__ import annotations

import math

import numpy as np

from . import fem

GUARD_Q = 1e-20
INV_2SQRT2 = 1.0 / (2.0 * math.sqrt(2.0))


def anisotropy(prm, p):
    """a(p) and da/dp (list) of Eq. (gs), with the small-gradient guard."""
    eps = prm.eps4
    q = sum(pi * pi for pi in p)
    guard = np.real(q) < GUARD_Q
    qs = np.where(guard, 1.0, q)
    s = sum(pi ** 4 for pi in p)
    a = 1.0 - 3.0 * eps + 4.0 * eps * s / qs ** 2
    dadp = [16.0 * eps * (pi ** 3 / qs ** 2 - s * pi / qs ** 3) for pi in p]
    a = np.where(guard, 1.0 + 0.0 * q, a)
    dadp = [np.where(guard, 0.0 * pi, d) for pi, d in zip(p, dadp)]
    return a, dadp, q, guard


def spatial(prm, phi, u, p, g, G4):
    """Level-wise spatial integrands: bulk source (psi part of R_phi), f_phi, D q(phi) grad u."""
    a, dadp, q, guard = anisotropy(prm, p)
    W2 = prm.W0 * prm.W0
    f_phi = [W2 * (a * a * pi + q * a * di) for pi, di in zip(p, dadp)]
    bulk = phi - phi ** 3 - prm.lam * (1.0 - phi * phi) ** 2 * (u + G4)
    mob = prm.D * (1.0 - phi) / 2.0 if prm.model == 1 else prm.D + 0.0 * phi
    return -bulk, f_phi, [mob * gi for gi in g], (a, q, guard)


def pointwise(prm, dt, phi, u, p, g, phin, un, G4, pn=None, old=None, phihat_old=None):
    """Gauss-point integrands (s_phi, f_phi[dim], s_u, f_u[dim]).

    ``old`` = (phi^n, u^n, grad phi^n, grad u^n, G4^n) and ``phihat_old`` =
    (phi^n - phi^{n-1})/dt enter only when theta < 1.
    """
    k = prm.k
    th = prm.theta
    sb, f_phi, f_diff, (a, q, guard) = spatial(prm, phi, u, p, g, G4)
    dphidt = (phi - phin) / dt
    phihat = dphidt if (th == 1.0 or prm.phihat_form == 1) else th * dphidt + (1.0 - th) * phihat_old
    B = 1.0 + (1.0 - k) * u
    if prm.time_form == 0:
        time_phi = prm.tau0 * B * a * a * dphidt
    else:
        an, _, _, _ = anisotropy(prm, pn)
        Bn = 1.0 + (1.0 - k) * un
        time_phi = prm.tau0 * (B * a * a * phi - Bn * an * an * phin) / dt
    s_phi = time_phi + th * sb
    f_phi = [th * fi for fi in f_phi]
    f_u = [th * fi for fi in f_diff]
    if th != 1.0:
        sbo, fpo, fdo, _ = spatial(prm, *old)
        s_phi = s_phi + (1.0 - th) * sbo
        f_phi = [fi + (1.0 - th) * fo for fi, fo in zip(f_phi, fpo)]
        f_u = [fi + (1.0 - th) * fo for fi, fo in zip(f_u, fdo)]
    A = ((1.0 + k) - (1.0 - k) * phin) / 2.0
    s_u = A * (u - un) / dt - 0.5 * phihat * B
    if prm.model == 1:
        c = INV_2SQRT2 * prm.W0 * B * phihat
        if prm.jat_normalised:
            qs = np.where(guard, 1.0, q)
            inv = np.where(guard, 0.0, 1.0 / np.sqrt(qs))
            f_u = [fi + c * pi * inv for fi, pi in zip(f_u, p)]
        else:
            f_u = [fi + c * pi for fi, pi in zip(f_u, p)]
    return s_phi, f_phi, s_u, f_u


def frozen_gradient(prm, xlast, t_new):
    """G4 of Eq. (directional) along the last axis; zero for the pure metal."""
    if prm.model == 1 and prm.lT != 0.0:
        return (xlast - prm.zT - prm.Vp * t_new) / prm.lT
    return 0.0 * xlast


def element_residual(mesh, prm, elems, phi_e, u_e, phin_e, un_e, t_n, dt, source=None, phinm1_e=None):
    """Element contributions (E, 2, 2^dim): [:,0] to R_phi, [:,1] to R_u.

    ``phi_e`` etc. are nodal values per element (E, 2^dim); ``elems`` the
    per-axis element indices (dim, E). ``source(xs) -> (S_phi, S_u)`` is an
    optional manufactured-solution source subtracted as (S, psi_i).
    ``phinm1_e``: phi^{n-1} per element (theta < 1; default phi^n).
    """
    dim, h = mesh.dim, mesh.h
    t_new = t_n + dt
    origin = [mesh.x0, mesh.y0, mesh.z0][:dim]
    dtype = np.result_type(phi_e, u_e, phin_e, un_e, prm.eps4)
    out = np.zeros((phi_e.shape[0], 2, phi_e.shape[1]), dtype=dtype)
    for xi, wref in fem.gauss_rule(dim, fem.order(mesh)):
        N, G = fem.basis(dim, xi, h, fem.order(mesh))
        w = wref * h ** dim
        phi = phi_e @ N
        u = u_e @ N
        phin = phin_e @ N
        un = un_e @ N
        p = [phi_e @ G[d] for d in range(dim)]
        g = [u_e @ G[d] for d in range(dim)]
        need_pn = prm.time_form == 1 or prm.theta != 1.0
        pn = [phin_e @ G[d] for d in range(dim)] if need_pn else None
        xs = [origin[d] + (elems[d] + xi[d]) * h for d in range(dim)]
        G4 = frozen_gradient(prm, xs[-1], t_new)
        old = phihat_old = None
        if prm.theta != 1.0:
            gn = [un_e @ G[d] for d in range(dim)]
            old = (phin, un, pn, gn, frozen_gradient(prm, xs[-1], t_n))
            pm1 = phin_e if phinm1_e is None else phinm1_e
            phihat_old = (phin - pm1 @ N) / dt
        s_phi, f_phi, s_u, f_u = pointwise(prm, dt, phi, u, p, g, phin, un, G4, pn, old, phihat_old)
        if source is not None:
            S_phi, S_u = source(xs)
            s_phi = s_phi - S_phi
            s_u = s_u - S_u
        out[:, 0, :] += w * (s_phi[:, None] * N[None, :] + sum(f_phi[d][:, None] * G[d][None, :] for d in range(dim)))
        out[:, 1, :] += w * (s_u[:, None] * N[None, :] + sum(f_u[d][:, None] * G[d][None, :] for d in range(dim)))
    return out


def gather(mesh, U, conn):
    n = mesh.n_nodes
    return U[:n][conn], U[n:][conn]


def residual(mesh, prm, U, Un, t_n, dt, source=None, chunk=1 << 18, Unm1=None):
    """Global residual F(U) (2 N_nodes,), field-major [R_phi ; R_u]; t_n is the time of U^n.

    ``Unm1`` is U^{n-1} (theta < 1 only; default U^n)."""
    n = mesh.n_nodes
    dtype = np.result_type(U, Un, prm.eps4)
    F = np.zeros(2 * n, dtype=dtype)
    elems_all = fem.all_elements(mesh)
    E = elems_all.shape[1]
    for s in range(0, E, chunk):
        elems = elems_all[:, s:s + chunk]
        conn = fem.connectivity(mesh, elems)
        phi_e, u_e = gather(mesh, U, conn)
        phin_e, un_e = gather(mesh, Un, conn)
        pm1_e = gather(mesh, Unm1, conn)[0] if Unm1 is not None else None
        c = element_residual(mesh, prm, elems, phi_e, u_e, phin_e, un_e, t_n, dt, source, pm1_e)
        F[:n] += fem.scatter_add(n, conn, c[:, 0, :])
        F[n:] += fem.scatter_add(n, conn, c[:, 1, :])
    return F


def residual_at_nodes(mesh, prm, U, Un, t_n, dt, nodes):
    """(R_phi, R_u) at the listed nodes only, from their adjacent elements."""
    nodes = np.asarray(nodes, dtype=np.int64)
    elems = fem.elements_of_nodes(mesh, nodes)
    conn = fem.connectivity(mesh, elems)
    phi_e, u_e = gather(mesh, U, conn)
    phin_e, un_e = gather(mesh, Un, conn)
    c = element_residual(mesh, prm, elems, phi_e, u_e, phin_e, un_e, t_n, dt)
    pos = {int(v): i for i, v in enumerate(nodes)}
    Rp = np.zeros(len(nodes), dtype=c.dtype)
    Ru = np.zeros(len(nodes), dtype=c.dtype)
    for e in range(conn.shape[0]):
        for a in range(conn.shape[1]):
            i = pos.get(int(conn[e, a]))
            if i is not None:
                Rp[i] += c[e, 0, a]
                Ru[i] += c[e, 1, a]
    return Rp, Ru
