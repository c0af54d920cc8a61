"""Newton-Krylov solution of F(U) = 0 for one implicit time step (Sec. 2.2, 2.3).

* Newton update U <- U + Lambda dU with backtracking: Lambda = 1, halved until
  ||F(U + Lambda dU)|| <= ||F(U)||, at most ``linesearch_max`` halvings
  (Eqs. newton-update, glob);
* stop when ||F|| < tau_r ||F0|| + tau_a (Eq. tolerance);
* inexact linear solves ||F' dU + F|| <= eta ||F|| with the forcing term
  eta_0 at l = 0 and, for l >= 1,
  eta_l = min(eta_max, max(gamma (||F_l||/||F_{l-1}||)^omega, gamma eta_{l-1}^omega, eta_min))
  (Eqs. force1..forcing; the printed eta_0 = 0.1 > eta_max = 0.01 is kept as
  the first value);
* restarted GMRES, right preconditioned (Eq. preJFmatvec), zero initial guess,
  modified Gram-Schmidt, Givens rotations; preconditioned directions are kept
  (flexible form) so an inexact preconditioner is allowed;
* the Jacobian action either by finite differences, Eq. (JFmatvec), with
  eps = sqrt((1 + ||U||) 2^-52) / ||v|| (the step "chosen heuristically" is read
  as this standard choice), or exactly (complex step);
* ``newton_direct``: Newton with a sparse direct solve of the exact Jacobian,
  used as the converged-solution reference.

Parity: pinned by convergence to the direct-solve solution and by the
invariants in tests/test_oracle_solver.py.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse.linalg as spla

from . import jacobian, precond
from .residual import residual

EPS_MACH = 2.0 ** -52


@dataclasses.dataclass
class StepStats:
    converged: bool = False
    newton_its: int = 0
    gmres_its: int = 0
    gmres_per_newton: list = dataclasses.field(default_factory=list)
    fnorm0: float = 0.0
    fnorm: float = 0.0
    linesearch_halvings: int = 0
    residual_evals: int = 0
    jv_evals: int = 0


def gmres(matvec, prec, b, tol_abs, restart, maxit):
    """Flexible right-preconditioned restarted GMRES (MGS) from x0 = 0. Returns (x, its, converged)."""
    n = b.shape[0]
    x = np.zeros(n)
    its = 0
    r = b.copy()
    beta = np.linalg.norm(r)
    resid = beta
    while beta > tol_abs and its < maxit:
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        m = 0
        for j in range(restart):
            Z[j] = prec(V[j])
            w = matvec(Z[j])
            its += 1
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            resid = abs(g[j + 1])
            m = j + 1
            if resid <= tol_abs or its >= maxit or H[j, j] == 0.0:
                break
        y = np.zeros(m)
        for i in range(m - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:m] @ y[i + 1:m]) / H[i, i]
        x = x + Z[:m].T @ y
        if resid <= tol_abs or its >= maxit:
            break
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        resid = beta
    return x, its, resid <= tol_abs


def forcing(prm, l, fnorm, fnorm_prev, eta_prev):
    if l == 0:
        return prm.eta0
    eta = prm.gamma * (fnorm / fnorm_prev) ** prm.omega
    eta = max(eta, prm.gamma * eta_prev ** prm.omega, prm.eta_min)
    return min(prm.eta_max, eta)


def fd_step(unorm, vnorm):
    """FD perturbation of Eq. (JFmatvec): sqrt((1 + ||U||) 2^-52) / ||v||."""
    return math.sqrt((1.0 + unorm) * EPS_MACH) / vnorm


def newton_step(mesh, prm, Un, t_n, dt, U0=None, exact=None, Unm1=None):
    """Solve F(U; U^n[, U^{n-1}]) = 0 by JFNK starting from U0 (default U^n). Returns (U, stats)."""
    U = (Un if U0 is None else U0).copy()
    exact = bool(prm.jvp_mode) if exact is None else exact
    F = residual(mesh, prm, U, Un, t_n, dt, Unm1=Unm1)
    st = StepStats(residual_evals=1)
    st.fnorm0 = st.fnorm = np.linalg.norm(F)
    tol = prm.newton_rtol * st.fnorm0 + prm.newton_atol
    eta_prev = prm.eta0
    fprev = None
    for l in range(prm.newton_maxit + 1):
        if st.fnorm < tol or st.fnorm == 0.0:
            st.converged = True
            break
        if l == prm.newton_maxit:
            break
        eta = forcing(prm, l, st.fnorm, fprev, eta_prev)
        M = precond.Preconditioner(mesh, prm, U, Un, dt)
        if exact:
            def mv(v, U=U):
                return jacobian.jvp(mesh, prm, U, Un, t_n, dt, v, Unm1=Unm1)
        else:
            unorm = np.linalg.norm(U)

            def mv(v, U=U, F=F, unorm=unorm):
                vn = np.linalg.norm(v)
                if vn == 0.0:
                    return np.zeros_like(v)
                e = fd_step(unorm, vn)
                return (residual(mesh, prm, U + e * v, Un, t_n, dt, Unm1=Unm1) - F) / e
        dU, its, _ = gmres(mv, M.apply, -F, eta * st.fnorm, prm.gmres_restart, prm.gmres_maxit)
        st.gmres_its += its
        st.gmres_per_newton.append(its)
        lam = 1.0
        accepted = False
        for _ in range(prm.linesearch_max + 1):
            Ut = U + lam * dU
            Ft = residual(mesh, prm, Ut, Un, t_n, dt, Unm1=Unm1)
            st.residual_evals += 1
            if np.linalg.norm(Ft) <= st.fnorm:
                accepted = True
                break
            lam *= 0.5
            st.linesearch_halvings += 1
        if not accepted:
            break
        fprev = st.fnorm
        eta_prev = eta
        U, F = Ut, Ft
        st.fnorm = np.linalg.norm(F)
        st.newton_its += 1
    return U, st


def newton_direct(mesh, prm, Un, t_n, dt, U0=None, rtol=1e-13, maxit=30, source=None, Unm1=None):
    """Newton with a sparse LU of the complex-step Jacobian; reference solution of F = 0.

    Returns (U, ||F||/||F0||). Backtracking as in Eq. (glob) guards the first steps.
    """
    U = (Un if U0 is None else U0).copy()
    F = residual(mesh, prm, U, Un, t_n, dt, source=source, Unm1=Unm1)
    f0 = np.linalg.norm(F)
    fn = f0
    for _ in range(maxit):
        if fn <= rtol * f0 or fn == 0.0:
            break
        J = jacobian.sparse_jacobian(mesh, prm, U, Un, t_n, dt, Unm1=Unm1)
        dU = spla.spsolve(J.tocsc(), -F)
        lam = 1.0
        for _ in range(30):
            Ft = residual(mesh, prm, U + lam * dU, Un, t_n, dt, source=source, Unm1=Unm1)
            if np.linalg.norm(Ft) <= fn:
                break
            lam *= 0.5
        U = U + lam * dU
        F = Ft
        fn = np.linalg.norm(F)
    return U, fn / f0 if f0 > 0 else 0.0


def run_steps(mesh, prm, U0, dt, nsteps, t0=0.0, direct=False):
    """nsteps theta-method steps (U^{-1} = U^0); returns (U_final, per-step stats or residual ratios)."""
    U = U0.copy()
    Uprev = U0.copy()
    t = t0
    hist = []
    for _ in range(nsteps):
        if direct:
            Unew, ratio = newton_direct(mesh, prm, U, t, dt, Unm1=Uprev)
            hist.append(ratio)
        else:
            Unew, st = newton_step(mesh, prm, U, t, dt, Unm1=Uprev)
            hist.append(st)
        Uprev, U = U, Unew
        t += dt
    return U, hist
