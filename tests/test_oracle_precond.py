"""Pins of the oracle preconditioner: textbook blocks, Galerkin coarsening, Chebyshev polynomial."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from synth import Mesh, Params
from oracle import precond as P
from tests import textbook as tb


@pytest.mark.parametrize("dim", [2, 3])
def test_blocks_with_uniform_state_are_textbook(dim):
    mesh = Mesh(dim, 4, 6, 2 if dim == 3 else 0, 0.7)
    n = mesh.n_nodes
    k, c, cu, cn = 0.15, 0.2, -0.6, -0.3
    prm = Params(model=1, k=k, eps4=0.05, tau0=1.3, W0=1.1, D=2.0, theta=1.0)
    U = np.concatenate([np.full(n, c), np.full(n, cu)])
    Un = np.concatenate([np.full(n, cn), np.zeros(n)])
    dt = 0.4
    M11, M22 = P.blocks(mesh, prm, U, Un, dt)
    M, K = tb.mass(mesh), tb.stiffness(mesh)
    # uniform phi: |grad phi| = 0, the guard sets a = 1
    W11 = prm.tau0 * (1 + (1 - k) * cu) / dt * M + prm.W0 ** 2 * K
    W22 = ((1 + k) - (1 - k) * cn) / 2 / dt * M + prm.D * (1 - c) / 2 * K
    assert abs(M11 - W11).max() < 1e-13 and abs(M22 - W22).max() < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_galerkin_coarse_operator_is_coarse_textbook(dim):
    """P^T A_h P equals the Q1 matrix of the coarse mesh (nested spaces, exact integration)."""
    mesh = Mesh(dim, 8, 4, 6 if dim == 3 else 0, 0.5)
    Pm = P.prolongation(mesh)
    cm = P.coarse_mesh(mesh)
    for A, Ac in ((tb.mass(mesh), tb.mass(cm)), (tb.stiffness(mesh), tb.stiffness(cm))):
        G = (Pm.T @ A @ Pm).tocsr()
        assert abs(G - Ac).max() < 1e-13 * abs(Ac).max()
    # P reproduces linear functions
    xs = tb.node_coords(cm)
    xf = tb.node_coords(mesh)
    f = 0.3 + sum((d + 1) * x for d, x in enumerate(xs))
    ff = 0.3 + sum((d + 1) * x for d, x in enumerate(xf))
    assert np.abs(Pm @ f - ff).max() < 1e-12


def _cheb_T(d, x):
    return np.cos(d * np.arccos(x)) if abs(x) <= 1 else np.cosh(d * np.arccosh(abs(x))) * (np.sign(x) ** d)


@pytest.mark.parametrize("degree", [1, 2, 3, 10])
def test_chebyshev_residual_polynomial(degree):
    """With A diagonal and D = I, x_deg = (1 - p(lam)) b / lam with p = T_d((theta-lam)/delta)/T_d(theta/delta)."""
    lam = np.linspace(0.05, 2.0, 40)
    A = sp.diags(lam).tocsr()
    b = np.linspace(1.0, 2.0, 40)
    lo, hi = 0.1, 1.9
    x = P.chebyshev(A, np.ones(40), b, None, lo, hi, degree)
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    p = np.array([_cheb_T(degree, (theta - l) / delta) for l in lam]) / _cheb_T(degree, theta / delta)
    assert np.abs(x - (1 - p) * b / lam).max() < 1e-12 * np.abs(b / lam).max()


def _blocks(name, dims):
    w = synth.scaled(synth.workload(name), *dims)
    U0 = synth.initial_state(w)
    return w, P.blocks(w.mesh, w.params, U0, U0, w.dt)


@pytest.mark.parametrize("name,dims", [("dendrite2d_1024", (32, 32)), ("alloy3d_256x256x128", (8, 8, 16))])
def test_vcycle_is_symmetric_and_convergent(name, dims):
    w, (M11, M22) = _blocks(name, dims)
    for A in (M11, M22):
        H = P.Hierarchy(w.mesh, A, 4)
        assert len(H.A) >= 3
        v = synth.uniform_pm1(1, A.shape[0])
        z = synth.uniform_pm1(2, A.shape[0])
        assert abs(v @ H.vcycle(z) - z @ H.vcycle(v)) < 1e-12 * np.abs(v) @ np.abs(H.vcycle(z))
        x = np.zeros_like(v)
        r0 = np.linalg.norm(v)
        for _ in range(6):
            x = x + H.vcycle(v - A @ x)
        assert np.linalg.norm(v - A @ x) < 0.7 ** 6 * r0
        # Gershgorin is an upper bound of the Jacobi-scaled spectrum
        d = A.diagonal()
        top = np.linalg.eigvalsh((A / np.sqrt(np.outer(d, d))).toarray()).max() if A.shape[0] < 3000 else None
        if top is not None:
            assert H.lmax[0] >= top - 1e-12


def test_jacobi_is_inverse_diagonal():
    w, (M11, M22) = _blocks("dendrite2d_128", (16, 16))
    U0 = synth.initial_state(w)
    pc = P.Preconditioner(w.mesh, w.params, U0, U0, w.dt)
    r = synth.uniform_pm1(3, 2 * w.mesh.n_nodes)
    n = w.mesh.n_nodes
    z = pc.apply(r)
    assert np.allclose(z[:n] * M11.diagonal(), r[:n], rtol=1e-15) and np.allclose(z[n:] * M22.diagonal(), r[n:], rtol=1e-15)
