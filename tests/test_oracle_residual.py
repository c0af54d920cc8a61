"""Pins of the oracle residual against what the paper and the mathematics fix.

* textbook Q1 mass / stiffness (Kronecker products of 1D matrices) where the
  residual is linear in the unknowns (Sec. 2.1.1 Galerkin form, Eqs. rpf..rtemp);
* the anisotropy a(n) of Eq. (gs) at its extreme directions (1 + eps along an
  axis, 1 - eps on a face diagonal, 1 - 5 eps/3 on the body diagonal);
* the anisotropic flux f = d/dp (W0^2 |p|^2 a^2 / 2), differentiated by sympy;
* the stationary flat interface phi = -tanh(n.x / (sqrt2 W0 a(n))) at u + G4 = 0
  (second-order consistency);
* the exact conservation identity of the solute / enthalpy equation;
* the published SplitMix64 sequence and the printed unknown counts / kappa values.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import synth
from synth import Mesh, Params
from oracle import residual as R
from tests import textbook as tb

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_splitmix64_published_sequence():
    want = [int(r[0], 16) for r in _read("splitmix64_seed0.txt")]
    assert synth.splitmix64_scalar(0, 4) == want
    assert [int(x) for x in synth.splitmix64(0, 4)] == want
    assert [int(x) for x in synth.splitmix64(987654321, 50)] == synth.splitmix64_scalar(987654321, 50)
    u = synth.uniform_pm1(3, 10000)
    assert u.min() >= -1.0 and u.max() < 1.0


def test_unknown_counts_match_paper():
    for nx, ny, nz, unk in _read("unknown_counts.txt"):
        nz = int(nz)
        m = Mesh(3 if nz else 2, int(nx), int(ny), nz, 1.0)
        assert m.n_dofs == int(unk)


def test_kappa_values_match_paper():
    a2, lam, k, h = 0.6267, 10.0, 0.14, 0.8
    D0 = a2 * lam / (1.0 + k)
    for mult, kap in _read("kappa_alloy.txt"):
        dt = float(mult) * 10.0 / 1024.0
        assert abs(2.0 * dt * D0 / h ** 2 / float(kap) - 1.0) < 3e-4


MESHES = [Mesh(2, 7, 5, 0, 0.7, 0.3, -0.2), Mesh(3, 4, 3, 5, 0.9, 0.1, 0.2, -0.3)]


@pytest.mark.parametrize("mesh", MESHES, ids=["2d", "3d"])
def test_pure_metal_u_equation_is_textbook(mesh):
    """Pure metal: R_u = M (u-u^n)/dt + D K u - M (phi-phi^n)/(2 dt), exactly linear."""
    prm = Params(model=0, eps4=0.05, lam=3.19, D=1.7)
    U, Un = synth.random_fields(mesh, 11)
    dt = 0.37
    n = mesh.n_nodes
    F = R.residual(mesh, prm, U, Un, 0.0, dt)
    M, K = tb.mass(mesh), tb.stiffness(mesh)
    want = M @ (U[n:] - Un[n:]) / dt + prm.D * (K @ U[n:]) - M @ (U[:n] - Un[:n]) / (2 * dt)
    assert np.abs(F[n:] - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("mesh", MESHES, ids=["2d", "3d"])
@pytest.mark.parametrize("jat", [0, 1])
def test_alloy_constant_phase_is_textbook(mesh, jat):
    """Alloy with constant phi, phi^n: grad phi = 0, so the antitrapping current vanishes and
    R_u = A(c_n) M (u-u^n)/dt + D (1-c)/2 K u - (c-c_n)/(2dt) M B(u); R_phi is a mass product."""
    k, c, cn = 0.15, 0.3, -0.4
    prm = Params(model=1, k=k, eps4=0.02, lam=2.5, D=2.0, lT=50.0, Vp=0.3, zT=-4.0, jat_normalised=jat)
    n = mesh.n_nodes
    _, Un = synth.random_fields(mesh, 5)
    U = np.concatenate([np.full(n, c), synth.uniform_pm1(9, n)])
    Un = np.concatenate([np.full(n, cn), Un[n:]])
    dt, tn = 0.25, 1.5
    F = R.residual(mesh, prm, U, Un, tn, dt)
    M, K = tb.mass(mesh), tb.stiffness(mesh)
    u, un = U[n:], Un[n:]
    A = ((1 + k) - (1 - k) * cn) / 2
    B = 1 + (1 - k) * u
    want_u = A * (M @ (u - un)) / dt + prm.D * (1 - c) / 2 * (K @ u) - (c - cn) / (2 * dt) * (M @ B)
    assert np.abs(F[n:] - want_u).max() <= 1e-13 * np.abs(want_u).max()
    # frozen gradient is linear in the last coordinate, so exact as a nodal Q1 field
    xl = tb.node_coords(mesh)[-1]
    g4 = (xl - prm.zT - prm.Vp * (tn + dt)) / prm.lT
    want_p = (c - cn) / dt * (M @ B) - (M @ np.full(n, c - c ** 3)) + prm.lam * (1 - c * c) ** 2 * (M @ (u + g4))
    assert np.abs(F[:n] - want_p).max() <= 1e-13 * np.abs(want_p).max()


@pytest.mark.parametrize("dim,p,a_want", [
    (2, (1.3, 0.0), lambda e: 1 + e),
    (2, (0.0, -0.8), lambda e: 1 + e),
    (2, (0.7, 0.7), lambda e: 1 - e),
    (3, (0.5, 0.5, 0.0), lambda e: 1 - e),
    (3, (0.4, -0.4, 0.4), lambda e: 1 - 5 * e / 3),
    (3, (0.0, 0.0, 2.0), lambda e: 1 + e),
])
def test_time_term_carries_anisotropy_squared(dim, p, a_want):
    """Shifting phi^n by a constant delta changes R_phi by tau0 a(n)^2 delta/dt M 1 (Eq. gs extremes)."""
    mesh = Mesh(dim, 4, 3, 3 if dim == 3 else 0, 0.6)
    eps = 0.05
    prm = Params(model=0, eps4=eps, tau0=1.7)
    xs = tb.node_coords(mesh)
    n = mesh.n_nodes
    phi = sum(pi * x for pi, x in zip(p, xs)) * 0.1
    U = np.concatenate([phi, np.zeros(n)])
    delta, dt = 0.01, 0.3
    Un1 = U.copy()
    Un2 = U.copy()
    Un2[:n] -= delta
    dF = R.residual(mesh, prm, U, Un2, 0.0, dt)[:n] - R.residual(mesh, prm, U, Un1, 0.0, dt)[:n]
    want = prm.tau0 * a_want(eps) ** 2 * delta / dt * (tb.mass(mesh) @ np.ones(n))
    assert np.abs(dF - want).max() <= 1e-12 * np.abs(want).max()


def _sympy_flux(p, eps, W0):
    """f(p) = d/dP [W0^2 |P|^2 a(P)^2 / 2] at P = p, differentiated symbolically."""
    import sympy as s

    P = s.symbols("p0:%d" % len(p), real=True)
    q = sum(x ** 2 for x in P)
    a = 1 - 3 * eps + 4 * eps * sum(x ** 4 for x in P) / q ** 2
    e = W0 ** 2 * q * a ** 2 / 2
    return np.array([float(s.diff(e, x).subs(dict(zip(P, p)))) for x in P])


@pytest.mark.parametrize("dim,p", [(2, (0.31, -0.72)), (3, (0.3, -0.7, 0.45))])
def test_anisotropic_flux_matches_energy_derivative(dim, p):
    """For linear phi the flux f(p) is constant; its eps-dependence shows up only at boundary
    nodes, as -f_d h^(dim-1) on the low face and +f_d h^(dim-1) on the high face of axis d."""
    mesh = Mesh(dim, 4, 5, 3 if dim == 3 else 0, 0.8, 1.0, -2.0, 0.5)
    n = mesh.n_nodes
    xs = tb.node_coords(mesh)
    phi = sum(pi * x for pi, x in zip(p, xs))
    U = np.concatenate([phi, 0.1 * np.ones(n)])
    W0 = 1.3
    e1, e2 = 0.07, 0.0
    F1 = R.residual(mesh, Params(model=0, eps4=e1, W0=W0), U, U, 0.0, 0.5)[:n]
    F2 = R.residual(mesh, Params(model=0, eps4=e2, W0=W0), U, U, 0.0, 0.5)[:n]
    df = _sympy_flux(p, e1, W0) - _sympy_flux(p, e2, W0)
    ijk = tb.node_ijk(mesh)
    nmax = [mesh.nx, mesh.ny, mesh.nz][:dim]
    interior = np.ones(n, dtype=bool)
    for d in range(dim):
        interior &= (ijk[d] > 0) & (ijk[d] < nmax[d])
    assert np.abs((F1 - F2)[interior]).max() < 1e-13
    for d in range(dim):
        face = (ijk[d] == 0)
        for e in range(dim):
            if e != d:
                face &= (ijk[e] > 0) & (ijk[e] < nmax[e])
        assert np.allclose((F1 - F2)[face], -df[d] * mesh.h ** (dim - 1), rtol=1e-12, atol=1e-14)


def _front_residual(dim, nel, angle_vec, eps, model=0):
    L = 12.0
    h = 2 * L / nel
    mesh = Mesh(dim, nel, nel, nel if dim == 3 else 0, h, -L, -L, -L)
    n = mesh.n_nodes
    xs = tb.node_coords(mesh)
    nv = np.array(angle_vec, float)
    nv /= np.linalg.norm(nv)
    s = sum(c * x for c, x in zip(nv, xs))
    q = (nv ** 2).sum()
    a = 1 - 3 * eps + 4 * eps * (nv ** 4).sum() / q ** 2
    phi = -np.tanh(s / (math.sqrt(2.0) * a))
    if model == 0:
        prm = Params(model=0, eps4=eps, lam=3.0)
        u = np.zeros(n)
    else:
        prm = Params(model=1, k=0.15, eps4=eps, lam=3.0, D=2.0, lT=40.0, Vp=0.5, zT=1.0)
        t_new = 0.2
        u = -(xs[-1] - prm.zT - prm.Vp * t_new) / prm.lT
    U = np.concatenate([phi, u])
    F = R.residual(mesh, prm, U, U, 0.0, 0.2)[:n]
    ijk = tb.node_ijk(mesh)
    inner = np.ones(n, dtype=bool)
    for d in range(dim):
        inner &= (ijk[d] >= nel // 4) & (ijk[d] <= 3 * nel // 4)
    return np.abs(F[inner]).max() / h ** dim


@pytest.mark.parametrize("dim,vec,eps,model", [
    (2, (1, 0), 0.0, 0),
    (2, (1, 0), 0.05, 0),
    (2, (1, 1), 0.05, 0),
    (2, (2, 1), 0.05, 0),
    (3, (1, 0, 0), 0.05, 1),
    (3, (1, 1, 1), 0.05, 0),
])
def test_flat_interface_is_stationary_to_second_order(dim, vec, eps, model):
    # nodal residual / h^dim in the interior halves of the box: O(h^2) (ratio -> 4)
    nel = [48, 96] if dim == 2 else [24, 48]
    e = [_front_residual(dim, m, vec, eps, model) for m in nel]
    assert e[0] / e[1] > (3.6 if dim == 2 else 3.2), e


@pytest.mark.parametrize("model,jat", [(0, 1), (1, 1), (1, 0)])
def test_conservation_identity(model, jat):
    """sum_i R_u,i = (1/dt) [ int Q(phi,u) - int Q(phi^n,u^n) ] with Q = u - phi/2 (pure metal)
    or Q = A(phi) B(u)/(1-k) (alloy); the flux terms drop because sum_i grad psi_i = 0."""
    mesh = Mesh(3, 3, 4, 3, 0.7)
    k = 1.0 if model == 0 else 0.15
    prm = Params(model=model, k=k, eps4=0.03, lam=2.0, D=2.0, jat_normalised=jat)
    U, Un = synth.random_fields(mesh, 17)
    n = mesh.n_nodes
    dt = 0.4
    F = R.residual(mesh, prm, U, Un, 0.0, dt)
    M = tb.mass(mesh)
    one = np.ones(n)
    if model == 0:
        I = lambda V: one @ (M @ (V[n:] - V[:n] / 2))
    else:
        I = lambda V: (((1 + k) - (1 - k) * V[:n]) / 2) @ (M @ (1 + (1 - k) * V[n:])) / (1 - k)
    assert abs(F[n:].sum() - (I(U) - I(Un)) / dt) < 1e-12 * np.abs(F[n:]).sum()


def test_guard_switches_off_anisotropy_and_antitrapping():
    """A uniform phase field has grad phi = 0 < 1e-20: R_u equals the run with the current off."""
    mesh = Mesh(2, 3, 3, 0, 1.0)
    n = mesh.n_nodes
    U = np.concatenate([np.full(n, 0.2), synth.uniform_pm1(1, n)])
    Un = np.concatenate([np.full(n, -0.1), synth.uniform_pm1(2, n)])
    p1 = Params(model=1, k=0.2, eps4=0.05, jat_normalised=1)
    p0 = Params(model=1, k=0.2, eps4=0.0, jat_normalised=0)
    F1 = R.residual(mesh, p1, U, Un, 0.0, 0.3)
    F0 = R.residual(mesh, p0, U, Un, 0.0, 0.3)
    assert np.abs(F1 - F0).max() < 1e-14


def test_residual_at_nodes_matches_full():
    mesh = Mesh(3, 5, 4, 3, 0.8)
    prm = Params(model=1, k=0.15, eps4=0.02, lam=3.1, D=2.0, lT=100.0, Vp=0.1)
    U, Un = synth.random_fields(mesh, 4)
    F = R.residual(mesh, prm, U, Un, 0.0, 0.2)
    nodes = np.array([0, 7, 33, mesh.n_nodes - 1])
    rp, ru = R.residual_at_nodes(mesh, prm, U, Un, 0.0, 0.2, nodes)
    n = mesh.n_nodes
    assert np.abs(rp - F[nodes]).max() < 1e-13 and np.abs(ru - F[n + nodes]).max() < 1e-13


def test_literal_time_form_differs_only_by_old_level_product():
    """time_form 1 = tau0 ([B a^2 phi]^{n+1} - [B a^2 phi]^n)/dt; with uniform phi^n (a^n = 1 by
    the guard) the difference to time_form 0 is tau0 (B - B^n) phi^n / dt integrated against psi."""
    mesh = Mesh(2, 4, 4, 0, 0.5)
    n = mesh.n_nodes
    U, _ = synth.random_fields(mesh, 8)
    Un = np.concatenate([np.full(n, 0.4), synth.uniform_pm1(12, n)])
    k = 0.3
    p0 = Params(model=1, k=k, eps4=0.04, time_form=0)
    p1 = dataclasses.replace(p0, time_form=1)
    dt = 0.5
    dF = R.residual(mesh, p1, U, Un, 0.0, dt)[:n] - R.residual(mesh, p0, U, Un, 0.0, dt)[:n]
    # time_form 1 - time_form 0 = tau0/dt [B a^2 phi - B^n phi^n - B a^2 (phi - phi^n)] = tau0/dt phi^n (B a^2 - B^n)
    # which is not a nodal product; check its u-independent part by two u^n values instead
    Un2 = Un.copy()
    Un2[n:] += 0.25
    dF2 = R.residual(mesh, p1, U, Un2, 0.0, dt)[:n] - R.residual(mesh, p0, U, Un2, 0.0, dt)[:n]
    want = -p0.tau0 / dt * 0.4 * (1 - k) * 0.25 * (tb.mass(mesh) @ np.ones(n))
    assert np.abs((dF2 - dF) - want).max() < 1e-13


@pytest.mark.parametrize("dim,p,norm", [(2, (0.4, -0.9), 1), (3, (0.3, 0.5, -0.6), 1), (3, (0.3, 0.5, -0.6), 0)])
def test_antitrapping_current_boundary_flux(dim, p, norm):
    """Linear phi shifted by delta in time, uniform u: phihat and j are uniform, so
    R_u = -phihat B/2 M 1 + j . int grad psi_i, i.e. -j_d h^(dim-1) on the low face of axis d
    (Eq. jat, entering F2 as +(j, grad psi_i) in Eq. conc2)."""
    mesh = Mesh(dim, 4, 3, 3 if dim == 3 else 0, 0.7)
    n = mesh.n_nodes
    k, W0, u0, delta, dt = 0.15, 1.2, -0.7, 0.05, 0.4
    prm = Params(model=1, k=k, W0=W0, eps4=0.02, D=2.0, jat_normalised=norm)
    xs = tb.node_coords(mesh)
    phi = sum(pi * x for pi, x in zip(p, xs)) * 0.2
    U = np.concatenate([phi, np.full(n, u0)])
    Un = np.concatenate([phi - delta, np.full(n, u0)])
    Fu = R.residual(mesh, prm, U, Un, 0.0, dt)[n:]
    B = 1 + (1 - k) * u0
    phihat = delta / dt
    rest = Fu + 0.5 * phihat * B * (tb.mass(mesh) @ np.ones(n))
    pv = 0.2 * np.array(p)
    j = W0 * B * phihat / (2 * math.sqrt(2)) * (pv / np.linalg.norm(pv) if norm else pv)
    ijk = tb.node_ijk(mesh)
    nmax = [mesh.nx, mesh.ny, mesh.nz][:dim]
    interior = np.ones(n, dtype=bool)
    for d in range(dim):
        interior &= (ijk[d] > 0) & (ijk[d] < nmax[d])
    assert np.abs(rest[interior]).max() < 1e-13
    for d in range(dim):
        for side, sgn in ((0, -1.0), (nmax[d], 1.0)):
            face = ijk[d] == side
            for e in range(dim):
                if e != d:
                    face &= (ijk[e] > 0) & (ijk[e] < nmax[e])
            assert np.allclose(rest[face], sgn * j[d] * mesh.h ** (dim - 1), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("theta", [0.5, 0.25])
def test_theta_method_linear_parts_are_textbook(theta):
    """Pure metal, theta-method (Eqs. dc, theta): R_u = M (u - u^n)/dt + theta D K u +
    (1 - theta) D K u^n - M phihat / 2, phihat = theta (phi - phi^n)/dt + (1 - theta)(phi^n - phi^{n-1})/dt."""
    mesh = Mesh(2, 6, 5, 0, 0.8)
    prm = Params(model=0, eps4=0.05, lam=3.0, D=1.3, theta=theta, phihat_form=0)
    U, Un = synth.random_fields(mesh, 31)
    Unm1 = synth.random_vector(mesh, 32)
    n = mesh.n_nodes
    dt = 0.3
    F = R.residual(mesh, prm, U, Un, 0.0, dt, Unm1=Unm1)
    M, K = tb.mass(mesh), tb.stiffness(mesh)
    phihat = theta * (U[:n] - Un[:n]) / dt + (1 - theta) * (Un[:n] - Unm1[:n]) / dt
    want = M @ (U[n:] - Un[n:]) / dt + prm.D * (K @ (theta * U[n:] + (1 - theta) * Un[n:])) - 0.5 * (M @ phihat)
    assert np.abs(F[n:] - want).max() <= 1e-13 * np.abs(want).max()
    # theta = 1 ignores U^{n-1}
    p1 = dataclasses.replace(prm, theta=1.0)
    assert np.array_equal(R.residual(mesh, p1, U, Un, 0.0, dt, Unm1=Unm1), R.residual(mesh, p1, U, Un, 0.0, dt))
