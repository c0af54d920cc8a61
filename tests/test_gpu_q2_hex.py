"""Triquadratic (Q2 hex, 3 x 3 x 3 Gauss) GPU kernels through the C-ABI against the CPU oracle.

Same bars as the Q1 and 2D Q2 parity tests: residual, tangent, adjoint,
(dF/dU^n)^T w and dF/d eps4 within 1e-12 normwise relative; point Jacobi within
1e-13 (FP64) or 1e-7 (FP32 reciprocal); multigrid within 1e-10 (FP64) or 2e-4
(FP32); converged time steps within 1e-8.
Meshes are ragged against the 4 x 2 x 2 element tile and include a single
element.
"""
import dataclasses

import numpy as np
import pytest

import synth
from synth import Mesh, Params
from oracle import jacobian as OJ
from oracle import precond as OP
from oracle import residual as OR
from oracle import solver as OS
from tests.gpu_util import dev, handle, host, rel

pytestmark = pytest.mark.gpu

PURE = Params(model=0, eps4=0.05, lam=3.19, D=2.0, precond=1)
ALLOY = Params(model=1, k=0.15, eps4=0.02, lam=3.1913, D=2.0, lT=60.0, Vp=0.12, zT=-5.0, precond=1)

CASES = [
    ("hex-pure-ragged", Mesh(3, 9, 5, 3, 0.9, -3.0, 1.0, 0.5, order=2), PURE),
    ("hex-alloy-ragged", Mesh(3, 7, 3, 5, 0.8, order=2), ALLOY),
    ("hex-alloy-jat0-literal", Mesh(3, 5, 4, 3, 0.8, order=2),
     dataclasses.replace(ALLOY, jat_normalised=0, time_form=1)),
    ("hex-pure-literal-time", Mesh(3, 4, 4, 4, 1.1, order=2), dataclasses.replace(PURE, time_form=1)),
    ("hex-1x1x1", Mesh(3, 1, 1, 1, 0.5, order=2), ALLOY),
    ("hex-2x3x5", Mesh(3, 2, 3, 5, 0.5, order=2), PURE),
]
IDS = [c[0] for c in CASES]


@pytest.mark.parametrize("name,mesh,prm", CASES, ids=IDS)
def test_q2_hex_residual_tangent_adjoint(name, mesh, prm):
    U, Un = synth.random_fields(mesh, 42)
    v = synth.random_vector(mesh, 8)
    w = synth.random_vector(mesh, 9)
    dt, tn = 0.37, 1.25
    h = handle(mesh, prm)
    assert h.n == mesh.n_dofs
    h.set_state(dev(Un), tn, dt)
    tU, tv, tw = dev(U), dev(v), dev(w)
    out = dev(np.zeros_like(U))
    h.residual(tU, out)
    assert rel(host(out), OR.residual(mesh, prm, U, Un, tn, dt)) <= 1e-12
    h.jvp(tU, tv, out)
    assert rel(host(out), OJ.jvp(mesh, prm, U, Un, tn, dt, v)) <= 1e-12
    h.jtvp(tU, tw, out)
    assert rel(host(out), OJ.jtvp(mesh, prm, U, Un, tn, dt, w)) <= 1e-12
    h.jtvp_prev(tU, tw, out)
    assert rel(host(out), OJ.dF_dUn_T(mesh, prm, U, Un, tn, dt, w)) <= 1e-12
    h.dFdp(tU, out, 0)
    assert rel(host(out), OJ.dF_deps4(mesh, prm, U, Un, tn, dt)) <= 1e-12
    h.jvp_fd(tU, tv, out)
    assert rel(host(out), OJ.jvp(mesh, prm, U, Un, tn, dt, v)) <= 1e-5


@pytest.mark.parametrize("form", [1, 0])
def test_q2_hex_theta_method(form):
    mesh = Mesh(3, 5, 3, 4, 0.9, order=2)
    prm = dataclasses.replace(ALLOY, theta=0.5, phihat_form=form)
    U, Un = synth.random_fields(mesh, 13)
    Unm1 = synth.random_vector(mesh, 14)
    v = synth.random_vector(mesh, 15)
    w = synth.random_vector(mesh, 16)
    dt, tn = 0.33, 0.9
    h = handle(mesh, prm)
    h.set_state(dev(Un), tn, dt)
    h.set_history(dev(Unm1))
    tU = dev(U)
    out = dev(np.zeros_like(U))
    h.residual(tU, out)
    assert rel(host(out), OR.residual(mesh, prm, U, Un, tn, dt, Unm1=Unm1)) <= 1e-12
    h.jvp(tU, dev(v), out)
    assert rel(host(out), OJ.jvp(mesh, prm, U, Un, tn, dt, v, Unm1=Unm1)) <= 1e-12
    h.jtvp(tU, dev(w), out)
    assert rel(host(out), OJ.jtvp(mesh, prm, U, Un, tn, dt, w, Unm1=Unm1)) <= 1e-12
    if form == 1:
        h.jtvp_prev(tU, dev(w), out)
        assert rel(host(out), OJ.dF_dUn_T(mesh, prm, U, Un, tn, dt, w)) <= 1e-12
        h.dFdp(tU, out, 0)
        assert rel(host(out), OJ.dF_deps4(mesh, prm, U, Un, tn, dt)) <= 1e-12


@pytest.mark.parametrize("prm", [PURE, ALLOY], ids=["pure", "alloy"])
@pytest.mark.parametrize("fp32,tol", [(0, 1e-13), (1, 1e-7)])
def test_q2_hex_jacobi_matches_oracle(prm, fp32, tol):
    mesh = Mesh(3, 7, 5, 3, 0.8, order=2)
    prm = dataclasses.replace(prm, smoother_fp32=fp32)
    U, Un = synth.random_fields(mesh, 21)
    Un = 0.5 * Un
    U = 0.5 * U
    h = handle(mesh, prm)
    h.set_state(dev(Un), 0.0, 0.3)
    h.precond_setup(dev(U))
    r = synth.random_vector(mesh, 11)
    z = dev(np.zeros_like(r))
    h.precond_apply(dev(r), z)
    want = OP.Preconditioner(mesh, prm, U, Un, 0.3).apply(r)
    assert rel(host(z), want) <= tol


@pytest.mark.parametrize("prm", [PURE, ALLOY], ids=["pure", "alloy"])
@pytest.mark.parametrize("fp32,tol", [(0, 1e-10), (1, 2e-4)])
@pytest.mark.parametrize("dims", [(6, 4, 4), (3, 5, 1), (1, 1, 1)], ids=["6x4x4", "3x5x1", "1x1x1"])
def test_q2_hex_multigrid_matches_oracle(prm, fp32, tol, dims):
    """Block Jacobi + multigrid for triquadratic hexes: 125-point stencils on the h/2 node
    lattice, the element-vertex level (the Galerkin product, filled directly from the same
    Gauss-point coefficients) and the trilinear levels below."""
    mesh = Mesh(3, dims[0], dims[1], dims[2], 0.8, order=2)
    prm = dataclasses.replace(prm, precond=2, smoother_fp32=fp32, mg_levels=4, cheb_degree=3)
    U, Un = synth.random_fields(mesh, 21)
    Un = 0.5 * Un
    U = 0.5 * U
    h = handle(mesh, prm)
    h.set_state(dev(Un), 0.0, 0.3)
    h.precond_setup(dev(U))
    r = synth.random_vector(mesh, 11)
    z = dev(np.zeros_like(r))
    h.precond_apply(dev(r), z)
    want = OP.Preconditioner(mesh, prm, U, Un, 0.3).apply(r)
    assert rel(host(z), want) <= tol


def test_q2_hex_residual_and_tangent_are_bitwise_deterministic():
    mesh = Mesh(3, 13, 7, 6, 0.8, order=2)
    U, Un = synth.random_fields(mesh, 3)
    v = synth.random_vector(mesh, 4)
    h = handle(mesh, ALLOY)
    h.set_state(dev(Un), 0.0, 0.2)
    tU, tv = dev(U), dev(v)
    ref = host(h.residual(tU, dev(np.zeros_like(U)))).copy()
    refj = host(h.jvp(tU, tv, dev(np.zeros_like(U)))).copy()
    F = dev(np.zeros_like(U))
    for _ in range(4):
        h.residual(tU, F)
        assert np.array_equal(host(F), ref)
        h.jvp(tU, tv, F)
        assert np.array_equal(host(F), refj)


HEX_STEPS = [
    ("pure-exact", PURE, dict(jvp_mode=1)),
    ("pure-fd", PURE, dict(jvp_mode=0)),
    ("alloy-exact-fp32", ALLOY, dict(jvp_mode=1, smoother_fp32=1)),
    ("pure-exact-gmg-fp32", PURE, dict(jvp_mode=1, precond=2, smoother_fp32=1, cheb_degree=3, gmres_maxit=30)),
]


@pytest.mark.parametrize("name,base,opts", HEX_STEPS, ids=[c[0] for c in HEX_STEPS])
def test_q2_hex_converged_steps_match_oracle(name, base, opts):
    mesh = Mesh(3, 5, 6, 4, 1.2, -3.0, -3.6, -2.4, order=2)
    prm = dataclasses.replace(base, **dict(dict(precond=1, smoother_fp32=0), **opts))
    U0 = synth.seed_state(mesh, prm, radius=2.5, centred=True)
    dt = 0.3
    h = handle(mesh, prm)
    h.set_state(dev(U0), 0.0, dt)
    Uo, t = U0.copy(), 0.0
    out = dev(np.zeros_like(U0))
    for _ in range(2):
        st = h.step()
        assert st["converged"], st
        Uo, ratio = OS.newton_direct(mesh, prm, Uo, t, dt)
        assert ratio < 1e-12
        t += dt
        assert rel(host(h.get_state(out)), Uo) <= 1e-8


def test_q2_hex_full_size_residual_on_sampled_nodes():
    """96^3 triquadratic elements (193^3 nodes, 14.4M dofs: the size of the 192^3 Q1 dendrite) on
    its [-76.8, 76.8]^3 box; the oracle evaluates sampled vertex, edge, face and cell nodes."""
    w = synth.workload("dendrite3d_192")
    mesh = dataclasses.replace(w.mesh, nx=96, ny=96, nz=96, h=2 * w.mesh.h, order=2)
    U0 = synth.seed_state(mesh, w.params, radius=10.0, centred=True)
    U = U0 + 0.05 * synth.uniform_pm1(77, mesh.n_dofs)
    h = handle(mesh, dataclasses.replace(w.params, precond=0))
    h.set_state(dev(U0), 1.0, w.dt)
    F = host(h.residual(dev(U), dev(np.zeros_like(U))))
    n = mesh.n_nodes
    nnx, nny = 2 * mesh.nx + 1, 2 * mesh.ny + 1
    picks = (synth.splitmix64(5, 40) % np.uint64(n)).astype(np.int64)
    fixed = [0, 1, nnx, nnx + 1, nnx * nny + nnx + 1, n - 1, n // 2]
    nodes = np.unique(np.concatenate([picks, fixed]))
    rp, ru = OR.residual_at_nodes(mesh, w.params, U, U0, 1.0, w.dt, nodes)
    scale = max(np.abs(rp).max(), np.abs(ru).max())
    assert np.abs(F[nodes] - rp).max() <= 1e-12 * scale
    assert np.abs(F[n + nodes] - ru).max() <= 1e-12 * scale


def test_q2_hex_adjoint_gradient_matches_oracle():
    """Discrete adjoint through 2 backward-Euler steps on a triquadratic box (point Jacobi):
    dS/d eps4 and dS/dU_0 against the oracle's direct-solve adjoint."""
    from oracle import adjoint as OA

    mesh = Mesh(3, 4, 4, 4, 2.0, order=2)
    prm = Params(model=0, eps4=0.04, lam=3.19, D=2.0, Delta=0.6, precond=1, jvp_mode=1, newton_rtol=1e-13,
                 smoother_fp32=0)
    U0 = synth.seed_state(mesh, prm, radius=5.0)
    dt, n = 0.5, 2
    states = OA.forward(mesh, prm, U0, 0.0, dt, n)
    w, _ = OA.solid_fraction_weights(mesh)
    g_eps, g0 = OA.gradient(mesh, prm, states, 0.0, dt, w)
    h = handle(mesh, prm)
    st = h.forward(dev(U0), 0.0, dt, n, 1)
    assert st["converged"]
    UN = host(h.get_state(dev(np.zeros_like(U0))))
    assert np.abs(UN - states[-1]).max() <= 1e-9 * np.abs(states[-1]).max()
    tg0 = dev(np.zeros_like(U0))
    ge, _, _ = h.adjoint(dev(w), None, tg0, rtol=1e-12)
    assert abs(ge - g_eps) <= 1e-7 * abs(g_eps)
    assert np.abs(host(tg0) - g0).max() <= 1e-7 * np.abs(g0).max()
