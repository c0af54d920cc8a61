"""Pins of the oracle's discrete adjoint against central differences of the forward solve."""
import dataclasses

import numpy as np

import synth
from synth import Mesh, Params
from oracle import adjoint as OA


def _S(mesh, prm, U0, dt, n):
    w, c = OA.solid_fraction_weights(mesh)
    return w @ OA.forward(mesh, prm, U0, 0.0, dt, n)[-1] + c


def test_solid_fraction_weights_integrate_exactly():
    mesh = Mesh(2, 5, 3, 0, 0.7)
    w, c = OA.solid_fraction_weights(mesh)
    n = mesh.n_nodes
    U = np.concatenate([np.ones(n), np.zeros(n)])  # phi = 1 everywhere: S = |Omega|
    assert abs(w @ U + c - 5 * 3 * 0.49) < 1e-12
    U[:n] = -1.0
    assert abs(w @ U + c) < 1e-12


def test_adjoint_gradient_matches_central_differences():
    mesh = Mesh(2, 10, 10, 0, 2.0)
    prm = Params(model=0, eps4=0.04, lam=3.19, D=2.0, Delta=0.6)
    dt, n = 0.5, 3
    U0 = synth.seed_state(mesh, prm, radius=6.0)
    states = OA.forward(mesh, prm, U0, 0.0, dt, n)
    w, _ = OA.solid_fraction_weights(mesh)
    g_eps, g0 = OA.gradient(mesh, prm, states, 0.0, dt, w)
    h = 1e-6
    fd = (_S(mesh, dataclasses.replace(prm, eps4=prm.eps4 + h), U0, dt, n)
          - _S(mesh, dataclasses.replace(prm, eps4=prm.eps4 - h), U0, dt, n)) / (2 * h)
    assert abs(g_eps - fd) <= 1e-5 * abs(fd)
    # Delta enters through u(x, 0) = -Delta only
    nn = mesh.n_nodes
    dU0 = np.concatenate([np.zeros(nn), -np.ones(nn)])
    pD = lambda d: synth.seed_state(mesh, dataclasses.replace(prm, Delta=d), radius=6.0)
    fdD = (_S(mesh, prm, pD(prm.Delta + h), dt, n) - _S(mesh, prm, pD(prm.Delta - h), dt, n)) / (2 * h)
    assert abs(g0 @ dU0 - fdD) <= 1e-5 * abs(fdD)


def test_alloy_adjoint_matches_central_differences():
    """Isothermal alloy (frozen gradient off) around a curved seed, antitrapping on."""
    mesh = Mesh(2, 10, 10, 0, 1.2, -6.0, -6.0)
    prm = Params(model=1, k=0.15, eps4=0.03, lam=3.19, D=2.0, Delta=0.5)
    dt, n = 0.3, 2
    U0 = synth.seed_state(mesh, prm, radius=3.0, centred=True)
    states = OA.forward(mesh, prm, U0, 0.0, dt, n)
    w, _ = OA.solid_fraction_weights(mesh)
    g_eps, g0 = OA.gradient(mesh, prm, states, 0.0, dt, w)
    h = 1e-5
    fd = (_S(mesh, dataclasses.replace(prm, eps4=prm.eps4 + h), U0, dt, n)
          - _S(mesh, dataclasses.replace(prm, eps4=prm.eps4 - h), U0, dt, n)) / (2 * h)
    assert abs(g_eps - fd) <= 1e-5 * abs(fd)
    nn = mesh.n_nodes
    dU0 = np.concatenate([np.zeros(nn), -np.ones(nn)])
    pD = lambda d: synth.seed_state(mesh, dataclasses.replace(prm, Delta=d), radius=3.0, centred=True)
    fdD = (_S(mesh, prm, pD(prm.Delta + h), dt, n) - _S(mesh, prm, pD(prm.Delta - h), dt, n)) / (2 * h)
    assert abs(g0 @ dU0 - fdD) <= 1e-5 * abs(fdD)


def test_q2_solid_fraction_weights_are_simpson():
    """Q2 interpolates phi = x^2 y exactly, so S = w^T U + c must equal the exact integral
    of (1 + x^2 y)/2 (trapezoid weights would not)."""
    mesh = Mesh(2, 3, 2, 0, 0.5, 1.0, 0.0, order=2)
    w, c = OA.solid_fraction_weights(mesh)
    xs, ys = np.meshgrid(*mesh.coords(), indexing="ij")
    phi = (xs ** 2 * ys).T.reshape(-1)
    U = np.concatenate([phi, np.zeros(mesh.n_nodes)])
    x0, x1, y0, y1 = 1.0, 2.5, 0.0, 1.0
    exact = 0.5 * ((x1 - x0) * (y1 - y0) + (x1 ** 3 - x0 ** 3) / 3 * (y1 ** 2 - y0 ** 2) / 2)
    assert abs(w @ U + c - exact) < 1e-13


def test_crank_nicolson_adjoint_matches_central_differences():
    """theta = 1/2 with phihat = (phi^{n+1} - phi^n)/dt: F_{n+1} depends on U_n also through the
    level-n spatial terms weighted 1 - theta; the adjoint recursion is unchanged (U_{n-1} does
    not enter), and dS/d eps4 picks up the level-n flux."""
    mesh = Mesh(2, 10, 10, 0, 1.2, -6.0, -6.0)
    prm = Params(model=1, k=0.15, eps4=0.03, lam=3.19, D=2.0, Delta=0.5, theta=0.5, phihat_form=1)
    dt, n = 0.3, 2
    U0 = synth.seed_state(mesh, prm, radius=3.0, centred=True)
    states = OA.forward(mesh, prm, U0, 0.0, dt, n)
    w, _ = OA.solid_fraction_weights(mesh)
    g_eps, g0 = OA.gradient(mesh, prm, states, 0.0, dt, w)
    h = 1e-5
    fd = (_S(mesh, dataclasses.replace(prm, eps4=prm.eps4 + h), U0, dt, n)
          - _S(mesh, dataclasses.replace(prm, eps4=prm.eps4 - h), U0, dt, n)) / (2 * h)
    assert abs(g_eps - fd) <= 1e-5 * abs(fd)
    nn = mesh.n_nodes
    dU0 = np.concatenate([np.zeros(nn), -np.ones(nn)])
    pD = lambda d: synth.seed_state(mesh, dataclasses.replace(prm, Delta=d), radius=3.0, centred=True)
    fdD = (_S(mesh, prm, pD(prm.Delta + h), dt, n) - _S(mesh, prm, pD(prm.Delta - h), dt, n)) / (2 * h)
    assert abs(g0 @ dU0 - fdD) <= 1e-5 * abs(fdD)
