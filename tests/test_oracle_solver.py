"""Pins of the oracle solver: GMRES, JFNK vs direct Newton, MMS order, invariants, symmetry, time order."""
import dataclasses
import math

import numpy as np
import pytest

import synth
from synth import Mesh, Params
from oracle import residual as R
from oracle import solver as S
from tests import textbook as tb


def test_gmres_solves_nonsymmetric_system():
    rng = np.random.default_rng(0)
    A = np.eye(60) * 4 + rng.standard_normal((60, 60)) * 0.3
    b = rng.standard_normal(60)
    x, its, ok = S.gmres(lambda v: A @ v, lambda v: v / 4.0, b, 1e-12 * np.linalg.norm(b), 10, 500)
    assert ok and np.abs(x - np.linalg.solve(A, b)).max() < 1e-10
    assert its > 10  # went through restarts


def test_forcing_terms():
    prm = Params()
    assert S.forcing(prm, 0, 1.0, None, None) == 0.1
    # gamma (ratio)^omega, floored by gamma eta^omega, capped at eta_max
    assert S.forcing(prm, 1, 1.0, 100.0, 0.1) == pytest.approx(0.01)
    assert S.forcing(prm, 2, 1e-9, 1e-3, 1e-5) == pytest.approx(max(0.9 * (1e-6) ** 1.5, 0.9 * (1e-5) ** 1.5, 1e-6))


@pytest.mark.parametrize("name,dims,pc,jv", [
    ("dendrite2d_128", (32, 32), 1, 0),
    ("dendrite2d_1024", (32, 32), 2, 1),
    ("alloy3d_256x256x128", (6, 6, 24), 2, 0),
    ("alloy3d_256x256x128", (6, 6, 24), 1, 1),
])
def test_jfnk_converges_to_direct_solution(name, dims, pc, jv):
    w = synth.scaled(synth.workload(name), *dims)
    prm = dataclasses.replace(w.params, precond=pc, jvp_mode=jv)
    U0 = synth.initial_state(w)
    U, st = S.newton_step(w.mesh, prm, U0, 0.0, w.dt)
    assert st.converged and st.fnorm < prm.newton_rtol * st.fnorm0
    Ud, ratio = S.newton_direct(w.mesh, prm, U0, 0.0, w.dt)
    assert ratio < 1e-12
    assert np.abs(U - Ud).max() <= 1e-8 * np.abs(Ud).max()


@pytest.mark.parametrize("model", [0, 1])
def test_conservation_over_steps(model):
    """Sum_i R_u,i is the exact difference quotient of the conserved integral, so after
    converged steps the integral changes by at most dt * sqrt(N) * ||F||."""
    if model == 0:
        w = synth.scaled(synth.workload("dendrite2d_128"), 24, 24)
        prm = w.params
    else:
        w = synth.scaled(synth.workload("alloy3d_256x256x128"), 4, 4, 24)
        prm = dataclasses.replace(w.params, precond=1)
    mesh, n = w.mesh, w.mesh.n_nodes
    M = tb.mass(mesh)
    k = prm.k
    if model == 0:
        I = lambda V: np.ones(n) @ (M @ (V[n:] - V[:n] / 2))
    else:
        I = lambda V: (((1 + k) - (1 - k) * V[:n]) / 2) @ (M @ (1 + (1 - k) * V[n:])) / (1 - k)
    U = synth.initial_state(w)
    t = 0.0
    for _ in range(2):
        Un = U
        U, st = S.newton_step(mesh, prm, Un, t, w.dt)
        assert st.converged
        bound = w.dt * math.sqrt(n) * st.fnorm
        assert abs(I(U) - I(Un)) <= bound * 1.001 + 1e-14 * abs(I(Un))
        t += w.dt


def test_centred_seed_keeps_square_symmetry():
    mesh = Mesh(2, 24, 24, 0, 1.5, -18.0, -18.0)
    prm = Params(model=0, eps4=0.05, lam=3.19, D=2.0, Delta=0.65, precond=1, jvp_mode=1)
    U = synth.seed_state(mesh, prm, radius=6.0, centred=True)
    t = 0.0
    for _ in range(2):
        U, st = S.newton_step(mesh, prm, U, t, 0.5)
        assert st.converged
        t += 0.5
    n = mesh.n_nodes
    for f in (U[:n], U[n:]):
        g = f.reshape(25, 25)  # [j, i]
        scale = np.abs(g).max()
        assert np.abs(g - g.T).max() < 1e-8 * scale
        assert np.abs(g - g[:, ::-1]).max() < 1e-8 * scale
        assert np.abs(g - g[::-1, :]).max() < 1e-8 * scale


def _mms_source(model, L, eps, lam, D, W0=1.0):
    import sympy as s

    x, y = s.symbols("x y", real=True)
    phi = s.Rational(6, 10) * s.cos(s.pi * x / L) + s.Rational(3, 10) * s.cos(s.pi * y / L)
    u = s.Rational(2, 10) * s.cos(s.pi * x / L) * s.cos(2 * s.pi * y / L) - s.Rational(2, 10)
    P0, P1 = s.symbols("P0 P1", real=True)
    q = P0 ** 2 + P1 ** 2
    a = 1 - 3 * eps + 4 * eps * (P0 ** 4 + P1 ** 4) / q ** 2
    e = W0 ** 2 * q * a ** 2 / 2
    sub = {P0: s.diff(phi, x), P1: s.diff(phi, y)}
    f = [s.diff(e, P0).subs(sub), s.diff(e, P1).subs(sub)]
    mob = D * (1 - phi) / 2 if model == 1 else D
    S_phi = -(s.diff(f[0], x) + s.diff(f[1], y)) - (phi - phi ** 3 - lam * (1 - phi ** 2) ** 2 * u)
    S_u = -(s.diff(mob * s.diff(u, x), x) + s.diff(mob * s.diff(u, y), y))
    fns = [s.lambdify((x, y), ex, "numpy") for ex in (S_phi, S_u, phi, u)]
    return fns


@pytest.mark.parametrize("model,eps", [(0, 0.0), (0, 0.05), (1, 0.05)])
def test_manufactured_solution_converges_second_order(model, eps):
    """Steady manufactured solution with zero-Neumann data; the sympy-derived source is added as
    (S, psi_i). The discrete nodal L2 error must fall by ~4 per halving of h (Q1, Sec. 2.1.1)."""
    L, lam, D = 4.0, 1.5, 2.0
    S_phi, S_u, phi_ex, u_ex = _mms_source(model, L, eps, lam, D)
    prm = Params(model=model, k=1.0 if model == 0 else 0.15, eps4=eps, lam=lam, D=D)
    errs = []
    for nel in (8, 16, 32):
        mesh = Mesh(2, nel, nel, 0, L / nel)
        xs = tb.node_coords(mesh)
        Uex = np.concatenate([phi_ex(*xs), u_ex(*xs)])
        src = lambda X: (S_phi(X[0], X[1]), S_u(X[0], X[1]))
        U, ratio = S.newton_direct(mesh, prm, Uex, 0.0, 1.0, U0=Uex, rtol=1e-12, source=src)
        errs.append(np.sqrt(mesh.h ** 2 * np.sum((U - Uex) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert r2 > 3.6 and r1 > 3.0, errs


@pytest.mark.slow
def test_backward_euler_is_first_order_in_time():
    mesh = Mesh(2, 10, 10, 0, 1.2)
    prm = Params(model=0, eps4=0.05, lam=3.19, D=2.0, Delta=0.65)
    U0 = synth.seed_state(mesh, prm, radius=5.0)
    T = 1.0
    ref, _ = S.run_steps(mesh, prm, U0, T / 256, 256, direct=True)
    errs = []
    for m in (8, 16, 32):
        U, _ = S.run_steps(mesh, prm, U0, T / m, m, direct=True)
        errs.append(np.linalg.norm(U - ref))
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.8 < errs[1] / errs[2] < 2.2, errs


@pytest.mark.slow
@pytest.mark.parametrize("form", [1, 0])
def test_crank_nicolson_temporal_order(form):
    """theta = 1/2 against a dt/256 reference: second order with phihat = (phi^{n+1} - phi^n)/dt
    (Sec. 4.1.2 reports second order for Crank-Nicolson); first order with the estimate printed
    as Eq. (theta), which is centred at t^n."""
    mesh = Mesh(2, 10, 10, 0, 1.2)
    prm = Params(model=0, eps4=0.05, lam=3.19, D=2.0, Delta=0.65, theta=0.5, phihat_form=form)
    U0 = synth.seed_state(mesh, prm, radius=5.0)
    T = 1.0
    ref, _ = S.run_steps(mesh, prm, U0, T / 256, 256, direct=True)
    errs = []
    for m in (8, 16, 32):
        U, _ = S.run_steps(mesh, prm, U0, T / m, m, direct=True)
        errs.append(np.linalg.norm(U - ref))
    r = [errs[0] / errs[1], errs[1] / errs[2]]
    if form == 1:
        assert r[0] > 3.3 and r[1] > 3.3, errs
    else:
        assert 1.7 < r[0] < 2.6 and 1.7 < r[1] < 2.6, errs
