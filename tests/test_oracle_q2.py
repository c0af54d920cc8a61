"""Pins of the biquadratic (Q2) elements with the 3x3 Gauss rule (Sec. 2.1.1, Sec. 4.1.3)."""
import dataclasses

import numpy as np
import pytest

import synth
from synth import Mesh, Params
from oracle import jacobian as J
from oracle import residual as R
from oracle import solver as S
from tests import textbook as tb
from tests.test_oracle_solver import _mms_source


def test_q2_node_layout_and_quadrature():
    m = Mesh(2, 3, 2, 0, 1.5, order=2)
    assert m.n_nodes == 7 * 5 and m.n_dofs == 70
    xs, ys = m.coords()
    assert np.allclose(xs, np.arange(7) * 0.75) and np.allclose(ys, np.arange(5) * 0.75)
    from oracle import fem

    rule = fem.gauss_rule(2, 2)
    assert len(rule) == 9 and abs(sum(w for _, w in rule) - 1.0) < 1e-15
    # the 3-point rule integrates x^5 exactly on [0,1]
    pts, wts = fem.gauss_1d(2)
    assert abs(sum(w * x ** 5 for x, w in zip(pts, wts)) - 1.0 / 6.0) < 1e-15


def test_q2_linear_u_equation_is_textbook():
    mesh = Mesh(2, 4, 3, 0, 0.9, 0.2, -0.4, order=2)
    prm = Params(model=0, eps4=0.05, lam=3.19, D=1.7)
    U, Un = synth.random_fields(mesh, 23)
    n = mesh.n_nodes
    dt = 0.37
    F = R.residual(mesh, prm, U, Un, 0.0, dt)
    M, K = tb.mass_q2(mesh), tb.stiffness_q2(mesh)
    want = M @ (U[n:] - Un[n:]) / dt + prm.D * (K @ U[n:]) - M @ (U[:n] - Un[:n]) / (2 * dt)
    assert np.abs(F[n:] - want).max() <= 1e-13 * np.abs(want).max()


def test_q2_jacobian_matches_central_differences():
    mesh = Mesh(2, 3, 3, 0, 0.8, order=2)
    prm = Params(model=1, k=0.15, eps4=0.03, lam=3.0, D=2.0, lT=30.0, Vp=0.1)
    U, Un = synth.random_fields(mesh, 4)
    v = synth.random_vector(mesh, 5)
    jv = J.jvp(mesh, prm, U, Un, 0.0, 0.4, v)
    h = 1e-6
    fd = (R.residual(mesh, prm, U + h * v, Un, 0.0, 0.4) - R.residual(mesh, prm, U - h * v, Un, 0.0, 0.4)) / (2 * h)
    assert np.abs(jv - fd).max() <= 1e-7 * np.abs(jv).max()
    w = synth.random_vector(mesh, 6)
    Js = J.sparse_jacobian(mesh, prm, U, Un, 0.0, 0.4)
    assert np.abs(Js.T @ w - J.jtvp(mesh, prm, U, Un, 0.0, 0.4, w)).max() <= 1e-12 * np.abs(Js.T @ w).max()


@pytest.mark.parametrize("model,eps", [(0, 0.0), (1, 0.0), (0, 0.05)])
def test_q2_manufactured_solution_converges_third_order(model, eps):
    """Q2 with the 3x3 Gauss rule on the steady manufactured solution of the Q1 test.

    Isotropic flux (eps4 = 0): the nodal L2 error falls by ~16 per halving of h
    (nodal superconvergence of Q2 on a tensor mesh; at least third order is asserted).
    With eps4 > 0 the flux W^2 a(n)^2 p + ... is homogeneous of degree 1 in p = grad(phi) but not
    differentiable at p = 0, and zero-Neumann data force grad(phi) = 0 at the box corners, so the
    source is only bounded there and the rate falls towards second order (ratios 7.4, 5.3, 4.5
    for nel 4..32); there only better-than-Q1 second order is asserted.
    """
    L, lam, D = 4.0, 1.5, 2.0
    S_phi, S_u, phi_ex, u_ex = _mms_source(model, L, eps, lam, D)
    prm = Params(model=model, k=1.0 if model == 0 else 0.15, eps4=eps, lam=lam, D=D)
    errs = []
    for nel in (4, 8, 16):
        mesh = Mesh(2, nel, nel, 0, L / nel, order=2)
        xs = tb.node_coords(mesh)
        Uex = np.concatenate([phi_ex(*xs), u_ex(*xs)])
        src = lambda X: (S_phi(X[0], X[1]), S_u(X[0], X[1]))
        U, ratio = S.newton_direct(mesh, prm, Uex, 0.0, 1.0, U0=Uex, rtol=1e-12, source=src)
        errs.append(np.sqrt((mesh.h / 2) ** 2 * np.sum((U - Uex) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    if eps == 0.0:
        assert r1 > 12.0 and r2 > 12.0, errs
    else:
        assert r1 > 4.5 and r2 > 4.5, errs


def test_q2_sampled_node_residual_matches_full_residual():
    """The one-node-at-a-time residual (used at full workload sizes) agrees with the full
    assembly on vertex, edge-midpoint and element-centre nodes of a Q2 box."""
    mesh = Mesh(2, 5, 4, 0, 0.7, 1.0, -2.0, order=2)
    prm = Params(model=1, k=0.15, eps4=0.02, lam=3.0, D=2.0, lT=40.0, Vp=0.1, zT=-3.0)
    U, Un = synth.random_fields(mesh, 31)
    F = R.residual(mesh, prm, U, Un, 0.4, 0.3)
    n = mesh.n_nodes
    nnx = 2 * mesh.nx + 1
    nodes = np.array([0, 1, 2, nnx, nnx + 1, 3 * nnx + 4, 5 * nnx + 7, n - 1, n - 2, n // 2])
    rp, ru = R.residual_at_nodes(mesh, prm, U, Un, 0.4, 0.3, nodes)
    assert np.abs(rp - F[nodes]).max() <= 1e-13 * np.abs(F).max()
    assert np.abs(ru - F[n + nodes]).max() <= 1e-13 * np.abs(F).max()


def test_q2_multigrid_hierarchy():
    """Q2 blocks on the h/2 node lattice: the first Galerkin product is the element-vertex Q1
    operator (9-point stencil, exact embedding of Q1 in Q2: P^T M_Q2 P of the mass block equals
    the Q1 mass matrix built from the same elements), and the V-cycle converges as a
    stationary iteration."""
    from oracle import precond as P

    mesh = Mesh(2, 8, 6, 0, 0.7, order=2)
    prm = Params(model=0, eps4=0.05, lam=3.19, D=2.0, precond=2)
    U, Un = synth.random_fields(mesh, 5)
    U, Un = 0.3 * U, 0.3 * Un
    M11, M22 = P.blocks(mesh, prm, U, Un, 0.4)
    lat = P.q2_lattice(mesh)
    Pm = P.prolongation(lat)
    # mass part of M22 for the pure metal is (1/dt) M: its Galerkin product is (1/dt) x Q1 mass
    q1 = Mesh(2, 8, 6, 0, 0.7)
    Mc = (Pm.T @ M22 @ Pm).tocsr()
    Kq1 = tb.mass(q1) / 0.4 + prm.theta * prm.D * tb.stiffness(q1)
    assert abs(Mc - Kq1).max() <= 1e-13 * abs(Kq1).max()
    # V-cycle as a stationary iteration on M11: contraction about 0.58 per cycle with degree-2
    # Chebyshev smoothing and 0.27 with degree 3 (the Q2 lattice mixes vertex, edge and centre
    # nodes, whose diagonals differ)
    rng = np.random.default_rng(0)
    b = rng.standard_normal(mesh.n_nodes)
    r0 = np.linalg.norm(b)
    for deg, bound in ((2, 1e-2), (3, 1e-5)):
        H = P.Hierarchy(lat, M11, 3, cheb_degree=deg)
        x = np.zeros_like(b)
        for _ in range(10):
            x = x + H.vcycle(b - M11 @ x)
        assert np.linalg.norm(b - M11 @ x) < bound * r0


# ---- triquadratic (Q2) hexahedra with the 3 x 3 x 3 Gauss rule ------------------------------

def _mms_source_3d(model, L, eps, lam, D, W0=1.0):
    """Steady manufactured solution on [0, L]^3 with zero-Neumann data and its sympy source."""
    import sympy as s

    x, y, z = s.symbols("x y z", real=True)
    X = (x, y, z)
    phi = (s.Rational(5, 10) * s.cos(s.pi * x / L) + s.Rational(3, 10) * s.cos(s.pi * y / L)
           + s.Rational(2, 10) * s.cos(s.pi * z / L))
    u = s.Rational(2, 10) * s.cos(s.pi * x / L) * s.cos(s.pi * y / L) * s.cos(s.pi * z / L) - s.Rational(2, 10)
    P = s.symbols("P0 P1 P2", real=True)
    q = P[0] ** 2 + P[1] ** 2 + P[2] ** 2
    a = 1 - 3 * eps + 4 * eps * (P[0] ** 4 + P[1] ** 4 + P[2] ** 4) / q ** 2
    e = W0 ** 2 * q * a ** 2 / 2
    sub = {P[d]: s.diff(phi, X[d]) for d in range(3)}
    f = [s.diff(e, P[d]).subs(sub) for d in range(3)]
    mob = D * (1 - phi) / 2 if model == 1 else D
    S_phi = -sum(s.diff(f[d], X[d]) for d in range(3)) - (phi - phi ** 3 - lam * (1 - phi ** 2) ** 2 * u)
    S_u = -sum(s.diff(mob * s.diff(u, X[d]), X[d]) for d in range(3))
    return [s.lambdify((x, y, z), ex, "numpy") for ex in (S_phi, S_u, phi, u)]


def test_q2_hex_node_layout_and_quadrature():
    m = Mesh(3, 3, 2, 4, 1.5, order=2)
    assert m.n_nodes == 7 * 5 * 9 and m.n_dofs == 2 * 315
    from oracle import fem

    rule = fem.gauss_rule(3, 2)
    assert len(rule) == 27 and abs(sum(w for _, w in rule) - 1.0) < 1e-15
    # x^5 y^4 z is integrated exactly by the tensor 3-point rule
    val = sum(w * xi[0] ** 5 * xi[1] ** 4 * xi[2] for xi, w in rule)
    assert abs(val - 1.0 / 60.0) < 1e-15


def test_q2_hex_linear_u_equation_is_textbook():
    """The u equation of the pure metal is linear: consistent Q2 mass and stiffness of the hex box,
    built as Kronecker products of the 1D quadratic element matrices."""
    mesh = Mesh(3, 3, 2, 2, 0.9, 0.2, -0.4, 0.3, order=2)
    prm = Params(model=0, eps4=0.05, lam=3.19, D=1.7)
    U, Un = synth.random_fields(mesh, 23)
    n = mesh.n_nodes
    dt = 0.37
    F = R.residual(mesh, prm, U, Un, 0.0, dt)
    M, K = tb.mass_q2(mesh), tb.stiffness_q2(mesh)
    want = M @ (U[n:] - Un[n:]) / dt + prm.D * (K @ U[n:]) - M @ (U[:n] - Un[:n]) / (2 * dt)
    assert np.abs(F[n:] - want).max() <= 1e-13 * np.abs(want).max()
    # row sums: the mass rows integrate 1 (|Omega|), the stiffness rows annihilate constants
    assert abs(M.sum() - 0.9 ** 3 * 3 * 2 * 2) < 1e-12 and np.abs(K @ np.ones(n)).max() < 1e-12


def test_q2_hex_jacobian_matches_central_differences():
    mesh = Mesh(3, 2, 2, 2, 0.8, order=2)
    prm = Params(model=1, k=0.15, eps4=0.03, lam=3.0, D=2.0, lT=30.0, Vp=0.1)
    U, Un = synth.random_fields(mesh, 4)
    v = synth.random_vector(mesh, 5)
    jv = J.jvp(mesh, prm, U, Un, 0.0, 0.4, v)
    h = 1e-6
    fd = (R.residual(mesh, prm, U + h * v, Un, 0.0, 0.4) - R.residual(mesh, prm, U - h * v, Un, 0.0, 0.4)) / (2 * h)
    assert np.abs(jv - fd).max() <= 1e-7 * np.abs(jv).max()
    w = synth.random_vector(mesh, 6)
    Js = J.sparse_jacobian(mesh, prm, U, Un, 0.0, 0.4)
    assert np.abs(Js.T @ w - J.jtvp(mesh, prm, U, Un, 0.0, 0.4, w)).max() <= 1e-12 * np.abs(Js.T @ w).max()
    assert np.abs(Js @ v - jv).max() <= 1e-12 * np.abs(jv).max()


@pytest.mark.parametrize("model", [0, 1])
def test_q2_hex_manufactured_solution_converges_fourth_order_at_nodes(model):
    """Triquadratic elements on a 3D steady manufactured solution with isotropic flux: the nodal
    L2 error falls by more than 12 per halving of h (measured 23 and 20 for nel 2 -> 4)."""
    L, lam, D = 4.0, 1.5, 2.0
    S_phi, S_u, phi_ex, u_ex = _mms_source_3d(model, L, 0.0, lam, D)
    prm = Params(model=model, k=1.0 if model == 0 else 0.15, eps4=0.0, lam=lam, D=D)
    errs = []
    for nel in (2, 4):
        mesh = Mesh(3, nel, nel, nel, L / nel, order=2)
        xs = tb.node_coords(mesh)
        Uex = np.concatenate([phi_ex(*xs), u_ex(*xs)])
        src = lambda X: (S_phi(X[0], X[1], X[2]), S_u(X[0], X[1], X[2]))
        U, ratio = S.newton_direct(mesh, prm, Uex, 0.0, 1.0, U0=Uex, rtol=1e-12, source=src)
        assert ratio <= 1e-11
        errs.append(np.sqrt((mesh.h / 2) ** 3 * np.sum((U - Uex) ** 2)))
    assert errs[0] / errs[1] > 12.0, errs


def test_q2_hex_sampled_node_residual_matches_full_residual():
    """One-node-at-a-time residual (the full-size GPU checks) against the full assembly on
    vertex, edge-, face- and cell-centre nodes of a Q2 hex box."""
    mesh = Mesh(3, 3, 2, 3, 0.7, 1.0, -2.0, 0.5, order=2)
    prm = Params(model=1, k=0.15, eps4=0.02, lam=3.0, D=2.0, lT=40.0, Vp=0.1, zT=-3.0)
    U, Un = synth.random_fields(mesh, 31)
    F = R.residual(mesh, prm, U, Un, 0.4, 0.3)
    n = mesh.n_nodes
    nnx, nny = 2 * mesh.nx + 1, 2 * mesh.ny + 1
    idx = lambda i, j, k: i + nnx * (j + nny * k)  # noqa: E731
    nodes = np.array([0, 1, idx(1, 1, 0), idx(1, 1, 1), idx(2, 2, 2), idx(3, 2, 1), idx(5, 3, 4), n - 1, n // 2])
    assert len(set(nodes.tolist())) == len(nodes)
    rp, ru = R.residual_at_nodes(mesh, prm, U, Un, 0.4, 0.3, nodes)
    assert np.abs(rp - F[nodes]).max() <= 1e-13 * np.abs(F).max()
    assert np.abs(ru - F[n + nodes]).max() <= 1e-13 * np.abs(F).max()


def test_q2_hex_multigrid_hierarchy():
    """Triquadratic blocks on the h/2 node lattice: the first Galerkin product is the trilinear
    operator of the element vertices (exact embedding of Q1 in Q2; for the pure metal M22 is
    (1/dt) M + theta D K, so the product equals the textbook Q1 matrices), and the V-cycle
    contracts as a stationary iteration."""
    from oracle import precond as P

    mesh = Mesh(3, 4, 2, 4, 0.7, order=2)
    prm = Params(model=0, eps4=0.05, lam=3.19, D=2.0, precond=2)
    U, Un = synth.random_fields(mesh, 5)
    U, Un = 0.3 * U, 0.3 * Un
    M11, M22 = P.blocks(mesh, prm, U, Un, 0.4)
    lat = P.q2_lattice(mesh)
    assert lat.n_nodes == mesh.n_nodes
    Pm = P.prolongation(lat)
    q1 = Mesh(3, 4, 2, 4, 0.7)
    Mc = (Pm.T @ M22 @ Pm).tocsr()
    Kq1 = tb.mass(q1) / 0.4 + prm.theta * prm.D * tb.stiffness(q1)
    assert abs(Mc - Kq1).max() <= 1e-13 * abs(Kq1).max()
    rng = np.random.default_rng(0)
    b = rng.standard_normal(mesh.n_nodes)
    r0 = np.linalg.norm(b)
    H = P.Hierarchy(lat, M11, 3, cheb_degree=3)
    x = np.zeros_like(b)
    for _ in range(10):
        x = x + H.vcycle(b - M11 @ x)
    assert np.linalg.norm(b - M11 @ x) < 1e-4 * r0
