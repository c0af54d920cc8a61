"""Q2 (biquadratic, 3 x 3 Gauss) GPU kernels through the C-ABI against the CPU oracle.

Same bars as the Q1 parity tests: residual, tangent, adjoint, (dF/dU^n)^T w and
dF/d eps4 within 1e-12 normwise relative; point Jacobi within 1e-13 (FP64
diagonal) or 1e-7 (FP32 reciprocal); converged time steps within 1e-8.
Meshes are ragged against the 16 x 8 element tile (partial tiles on both
axes) and include single-element boxes.
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
    ("q2-pure-ragged", Mesh(2, 37, 19, 0, 0.9, -3.0, 1.0, order=2), PURE),
    ("q2-alloy-ragged", Mesh(2, 35, 17, 0, 0.8, order=2), ALLOY),
    ("q2-alloy-jat0-literal", Mesh(2, 33, 9, 0, 0.8, order=2),
     dataclasses.replace(ALLOY, jat_normalised=0, time_form=1)),
    ("q2-pure-literal-time", Mesh(2, 18, 18, 0, 1.1, order=2), dataclasses.replace(PURE, time_form=1)),
    ("q2-1x1", Mesh(2, 1, 1, 0, 0.5, order=2), ALLOY),
    ("q2-2x3", Mesh(2, 2, 3, 0, 0.5, order=2), PURE),
]
IDS = [c[0] for c in CASES]


@pytest.mark.parametrize("name,mesh,prm", CASES, ids=IDS)
def test_q2_residual_tangent_adjoint(name, mesh, prm):
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
def test_q2_theta_method(form):
    mesh = Mesh(2, 21, 13, 0, 0.9, order=2)
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
def test_q2_jacobi_matches_oracle(prm, fp32, tol):
    mesh = Mesh(2, 19, 11, 0, 0.8, order=2)
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
@pytest.mark.parametrize("dims", [(24, 20), (3, 5), (1, 1)], ids=["24x20", "3x5", "1x1"])
def test_q2_multigrid_matches_oracle(prm, fp32, tol, dims):
    """Block Jacobi + multigrid for Q2: 25-point stencils on the h/2 node lattice, Galerkin
    coarsening to the element vertices and the Q1 levels below (odd element counts stop the
    hierarchy at the vertex grid; a single element has a 3 x 3 lattice and a 2 x 2 vertex grid)."""
    mesh = Mesh(2, dims[0], dims[1], 0, 0.8, order=2)
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


def test_q2_residual_is_bitwise_deterministic():
    mesh = Mesh(2, 45, 27, 0, 0.8, order=2)
    U, Un = synth.random_fields(mesh, 3)
    h = handle(mesh, ALLOY)
    h.set_state(dev(Un), 0.0, 0.2)
    tU = dev(U)
    ref = host(h.residual(tU, dev(np.zeros_like(U)))).copy()
    F = dev(np.zeros_like(U))
    for _ in range(5):
        h.residual(tU, F)
        assert np.array_equal(host(F), ref)


Q2_STEPS = [
    ("pure-exact", dict(jvp_mode=1)),
    ("pure-fd", dict(jvp_mode=0)),
    ("pure-exact-gmg", dict(jvp_mode=1, precond=2, cheb_degree=3, gmres_maxit=30)),
]


@pytest.mark.parametrize("name,opts", Q2_STEPS, ids=[c[0] for c in Q2_STEPS])
def test_q2_converged_steps_match_oracle(name, opts):
    w = synth.scaled(synth.workload("dendrite2d_128"), 16, 16)
    mesh = dataclasses.replace(w.mesh, order=2)
    prm = dataclasses.replace(w.params, **dict(dict(precond=1, smoother_fp32=0), **opts))
    U0 = synth.seed_state(mesh, prm, radius=8.0)
    h = handle(mesh, prm)
    h.set_state(dev(U0), 0.0, w.dt)
    Uo, t = U0.copy(), 0.0
    out = dev(np.zeros_like(U0))
    for _ in range(2):
        st = h.step()
        assert st["converged"], st
        Uo, ratio = OS.newton_direct(mesh, prm, Uo, t, w.dt)
        assert ratio < 1e-12
        t += w.dt
        assert rel(host(h.get_state(out)), Uo) <= 1e-8


def test_q2_alloy_step_matches_oracle():
    mesh = Mesh(2, 10, 14, 0, 0.8, order=2)
    prm = dataclasses.replace(ALLOY, jvp_mode=1, smoother_fp32=1)
    U0 = synth.seed_state(mesh, prm, radius=4.0)
    h = handle(mesh, prm)
    h.set_state(dev(U0), 0.0, 0.2)
    st = h.step()
    assert st["converged"], st
    Uo, ratio = OS.newton_direct(mesh, prm, U0, 0.0, 0.2)
    assert ratio < 1e-12
    assert rel(host(h.get_state(dev(np.zeros_like(U0)))), Uo) <= 1e-8


def test_q2_full_size_residual_on_sampled_nodes():
    """1024^2 Q2 elements (2049^2 nodes) on the dendrite2d_1024 box; the oracle evaluates sampled
    vertex, edge and centre nodes one by one."""
    w = synth.workload("dendrite2d_1024")
    mesh = dataclasses.replace(w.mesh, order=2)
    U0 = synth.seed_state(mesh, w.params, radius=8.0)
    U = U0 + 0.05 * synth.uniform_pm1(77, mesh.n_dofs)
    h = handle(mesh, dataclasses.replace(w.params, precond=0))
    h.set_state(dev(U0), 1.0, w.dt)
    F = host(h.residual(dev(U), dev(np.zeros_like(U))))
    n = mesh.n_nodes
    nnx = 2 * mesh.nx + 1
    picks = (synth.splitmix64(5, 48) % np.uint64(n)).astype(np.int64)
    nodes = np.unique(np.concatenate([picks, [0, 1, nnx, nnx + 1, n - 1, n // 2]]))
    rp, ru = OR.residual_at_nodes(mesh, w.params, U, U0, 1.0, w.dt, nodes)
    scale = max(np.abs(rp).max(), np.abs(ru).max())
    assert np.abs(F[nodes] - rp).max() <= 1e-12 * scale
    assert np.abs(F[n + nodes] - ru).max() <= 1e-12 * scale


@pytest.mark.parametrize("variant", ["be-jacobi", "cn-multigrid"])
def test_q2_adjoint_gradient_matches_oracle(variant):
    """Discrete adjoint through 3 steps on a Q2 box (Simpson solid-fraction weights): dS/d eps4
    and dS/dU_0 against the oracle's direct-solve adjoint; backward Euler with point Jacobi, and
    Crank-Nicolson with the lattice multigrid in the transposed solves."""
    from oracle import adjoint as OA

    mesh = Mesh(2, 8, 8, 0, 2.0, order=2)
    prm = Params(model=0, eps4=0.04, lam=3.19, D=2.0, Delta=0.6, precond=1, jvp_mode=1, newton_rtol=1e-13,
                 smoother_fp32=0)
    if variant == "cn-multigrid":
        prm = dataclasses.replace(prm, theta=0.5, phihat_form=1, precond=2, mg_levels=3)
    U0 = synth.seed_state(mesh, prm, radius=6.0)
    dt, n = 0.5, 3
    states = OA.forward(mesh, prm, U0, 0.0, dt, n)
    w, _ = OA.solid_fraction_weights(mesh)
    g_eps, g0 = OA.gradient(mesh, prm, states, 0.0, dt, w)
    h = handle(mesh, prm)
    st = h.forward(dev(U0), 0.0, dt, n, 2)
    assert st["converged"]
    UN = host(h.get_state(dev(np.zeros_like(U0))))
    assert np.abs(UN - states[-1]).max() <= 1e-9 * np.abs(states[-1]).max()
    tg0 = dev(np.zeros_like(U0))
    ge, _, _ = h.adjoint(dev(w), None, tg0, rtol=1e-12)
    assert abs(ge - g_eps) <= 1e-7 * abs(g_eps)
    assert np.abs(host(tg0) - g0).max() <= 1e-7 * np.abs(g0).max()
