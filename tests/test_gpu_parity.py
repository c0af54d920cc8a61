"""GPU kernels (through the C-ABI) against the CPU oracle on the same seeded inputs.

Tolerances: residual, tangent, adjoint and dF/d eps4 normwise 1e-12 relative
(FP64 kernels with a different summation order than the oracle); converged
time steps 1e-8 relative to the solution (Newton tolerance 1e-10 relative on
||F||, oracle solved to 1e-13 with a direct solver).
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
    ("2d-pure-ragged", Mesh(2, 37, 19, 0, 0.9, -3.0, 1.0), PURE),
    ("2d-alloy-ragged", Mesh(2, 35, 17, 0, 0.8), ALLOY),
    ("2d-alloy-jat0", Mesh(2, 33, 9, 0, 0.8), dataclasses.replace(ALLOY, jat_normalised=0)),
    ("2d-pure-literal-time", Mesh(2, 18, 18, 0, 1.1), dataclasses.replace(PURE, time_form=1)),
    ("3d-pure-ragged", Mesh(3, 19, 9, 6, 0.8, -1.0, 2.0, 0.5), PURE),
    ("3d-alloy-ragged", Mesh(3, 17, 10, 9, 0.8), ALLOY),
    ("3d-alloy-literal-jat0", Mesh(3, 9, 5, 5, 0.7), dataclasses.replace(ALLOY, time_form=1, jat_normalised=0)),
    ("2d-1x1", Mesh(2, 1, 1, 0, 0.5), ALLOY),
    ("2d-2x3", Mesh(2, 2, 3, 0, 0.5), PURE),
    ("3d-1x1x1", Mesh(3, 1, 1, 1, 0.5), ALLOY),
    ("3d-3x2x5", Mesh(3, 3, 2, 5, 0.6), PURE),
]
IDS = [c[0] for c in CASES]


def _inputs(mesh, seed=42):
    U, Un = synth.random_fields(mesh, seed)
    return U, Un


@pytest.mark.parametrize("name,mesh,prm", CASES, ids=IDS)
def test_residual_matches_oracle(name, mesh, prm):
    U, Un = _inputs(mesh)
    dt, tn = 0.37, 1.25
    h = handle(mesh, prm)
    h.set_state(dev(Un), tn, dt)
    tU = dev(U)
    F = dev(np.zeros_like(U))
    h.residual(tU, F)
    want = OR.residual(mesh, prm, U, Un, tn, dt)
    assert rel(host(F), want) <= 1e-12


@pytest.mark.parametrize("name,mesh,prm", CASES, ids=IDS)
def test_tangent_adjoint_and_parameter_derivative(name, mesh, prm):
    U, Un = _inputs(mesh, 7)
    v = synth.random_vector(mesh, 8)
    w = synth.random_vector(mesh, 9)
    dt, tn = 0.41, 0.5
    h = handle(mesh, prm)
    h.set_state(dev(Un), tn, dt)
    tU, tv, tw = dev(U), dev(v), dev(w)
    out = dev(np.zeros_like(U))
    h.jvp(tU, tv, out)
    assert rel(host(out), OJ.jvp(mesh, prm, U, Un, tn, dt, v)) <= 1e-12
    h.jtvp(tU, tw, out)
    assert rel(host(out), OJ.jtvp(mesh, prm, U, Un, tn, dt, w)) <= 1e-12
    h.jtvp_prev(tU, tw, out)
    assert rel(host(out), OJ.dF_dUn_T(mesh, prm, U, Un, tn, dt, w)) <= 1e-12
    h.dFdp(tU, out, 0)
    want = OJ.dF_deps4(mesh, prm, U, Un, tn, dt)
    assert rel(host(out), want) <= 1e-12
    # finite-difference action (Eq. JFmatvec) approximates the exact one
    h.jvp_fd(tU, tv, out)
    assert rel(host(out), OJ.jvp(mesh, prm, U, Un, tn, dt, v)) <= 1e-5


@pytest.mark.parametrize("name,mesh,prm", [
    ("2d-alloy", Mesh(2, 35, 17, 0, 0.8), ALLOY),
    ("3d-alloy-literal", Mesh(3, 17, 10, 9, 0.8), dataclasses.replace(ALLOY, time_form=1)),
    ("3d-pure", Mesh(3, 19, 9, 6, 0.8, -1.0, 2.0, 0.5), PURE),
], ids=["2d-alloy", "3d-alloy-literal", "3d-pure"])
def test_flat_phase_field_takes_the_zero_gradient_branch(name, mesh, prm):
    """phi = 1 (U and U^n) on the nodes with x index below 7: there grad phi is exactly zero at
    every Gauss point, and both sides take the anisotropy's guarded branch (a = 1, n = 0) for
    the residual, the tangent, the transposes and dF/d eps4."""
    U, Un = _inputs(mesh, 13)
    n = mesh.n_nodes
    flat = np.arange(n) % (mesh.nx + 1) < 7
    U[:n][flat] = 1.0
    Un[:n][flat] = 1.0
    v = synth.random_vector(mesh, 14)
    dt, tn = 0.37, 1.25
    h = handle(mesh, prm)
    h.set_state(dev(Un), tn, dt)
    tU, tv = dev(U), dev(v)
    out = dev(np.zeros_like(U))
    h.residual(tU, out)
    assert rel(host(out), OR.residual(mesh, prm, U, Un, tn, dt)) <= 1e-12
    h.jvp(tU, tv, out)
    assert rel(host(out), OJ.jvp(mesh, prm, U, Un, tn, dt, v)) <= 1e-12
    h.jtvp(tU, tv, out)
    assert rel(host(out), OJ.jtvp(mesh, prm, U, Un, tn, dt, v)) <= 1e-12
    h.jtvp_prev(tU, tv, out)
    assert rel(host(out), OJ.dF_dUn_T(mesh, prm, U, Un, tn, dt, v)) <= 1e-12
    h.dFdp(tU, out, 0)
    assert rel(host(out), OJ.dF_deps4(mesh, prm, U, Un, tn, dt)) <= 1e-12


def test_residual_is_bitwise_deterministic():
    mesh = Mesh(3, 21, 13, 9, 0.8)
    U, Un = _inputs(mesh, 3)
    h = handle(mesh, ALLOY)
    h.set_state(dev(Un), 0.0, 0.2)
    tU = dev(U)
    ref = host(h.residual(tU, dev(np.zeros_like(U)))).copy()
    F = dev(np.zeros_like(U))
    for _ in range(10):
        h.residual(tU, F)
        assert np.array_equal(host(F), ref)
    assert h.dot(tU, tU) == h.dot(tU, tU)
    assert abs(h.dot(tU, tU) - float(U @ U)) <= 1e-12 * float(U @ U)
    # the tangent and its transpose (tile-level sums in shared memory) repeat bitwise too
    tv = dev(synth.random_vector(mesh, 4))
    for op in (h.jvp, h.jtvp):
        ref = host(op(tU, tv, dev(np.zeros_like(U)))).copy()
        for _ in range(5):
            op(tU, tv, F)
            assert np.array_equal(host(F), ref)


def _precond_case(dim, fp32, kind=2):
    if dim == 2:
        w = synth.scaled(synth.workload("dendrite2d_1024"), 32, 32)
    elif dim == 3:
        w = synth.scaled(synth.workload("alloy3d_256x256x128"), 16, 16, 32)
    else:
        # 65 x 65 x 33 nodes: the finest level launches 1734 smoother blocks (the 8-blocks-per-SM
        # build), the 33 x 33 x 17 level 324 (the 3-blocks-per-SM build), the coarser ones fewer
        # than 297 (the 2-blocks-per-SM build)
        w = synth.scaled(synth.workload("alloy3d_256x256x128"), 64, 64, 32)
    prm = dataclasses.replace(w.params, precond=kind, smoother_fp32=fp32)
    U0 = synth.initial_state(w)
    U = U0 + 0.01 * synth.random_vector(w.mesh, 3)
    return w, prm, U, U0


@pytest.mark.parametrize("dim", [2, 3, "3d-64x64x32"])
@pytest.mark.parametrize("kind,fp32,tol", [(1, 0, 1e-13), (2, 0, 1e-10), (2, 1, 2e-4)])
def test_preconditioner_matches_oracle(dim, kind, fp32, tol):
    """Jacobi and the GMG V-cycle per block: FP64 operators to roundoff, FP32 to a few
    single-precision ulps amplified by the V-cycle (bound 2e-4 normwise)."""
    w, prm, U, U0 = _precond_case(dim, fp32, kind)
    h = handle(w.mesh, prm)
    h.set_state(dev(U0), 0.0, w.dt)
    h.precond_setup(dev(U))
    r = synth.random_vector(w.mesh, 11)
    z = dev(np.zeros_like(r))
    h.precond_apply(dev(r), z)
    want = OP.Preconditioner(w.mesh, prm, U, U0, w.dt).apply(r)
    assert rel(host(z), want) <= tol


STEP_CASES = [
    ("dendrite2d_128", (32, 32), dict(precond=1, jvp_mode=0, smoother_fp32=0), 2),
    ("dendrite2d_1024", (32, 32), dict(precond=2, jvp_mode=1, smoother_fp32=1), 2),
    ("dendrite3d_192", (12, 12, 12), dict(precond=2, jvp_mode=0, smoother_fp32=0), 1),
    ("alloy3d_256x256x128", (8, 8, 24), dict(precond=2, jvp_mode=1, smoother_fp32=1), 2),
    ("alloy3d_256x256x128", (8, 8, 24), dict(precond=2, jvp_mode=0, smoother_fp32=0), 1),
]


@pytest.mark.parametrize("name,dims,opts,nsteps", STEP_CASES,
                         ids=[f"{c[0]}-{'x'.join(map(str, c[1]))}-pc{c[2]['precond']}-jv{c[2]['jvp_mode']}-fp32{c[2]['smoother_fp32']}" for c in STEP_CASES])
def test_converged_steps_match_oracle(name, dims, opts, nsteps):
    w = synth.scaled(synth.workload(name), *dims)
    prm = dataclasses.replace(w.params, **opts)
    U0 = synth.initial_state(w)
    h = handle(w.mesh, prm)
    h.set_state(dev(U0), 0.0, w.dt)
    Uo = U0.copy()
    t = 0.0
    out = dev(np.zeros_like(U0))
    for _ in range(nsteps):
        st = h.step()
        assert st["converged"] and st["fnorm"] < prm.newton_rtol * st["fnorm0"], st
        Uo, ratio = OS.newton_direct(w.mesh, prm, Uo, t, w.dt)
        assert ratio < 1e-12
        t += w.dt
        assert rel(host(h.get_state(out)), Uo) <= 1e-8
    assert abs(h.time - t) < 1e-12


SMALL_SYSTEMS = [
    ("2d-2x2-alloy", Mesh(2, 2, 2, 0, 0.7), ALLOY),
    ("3d-1x1x1-pure", Mesh(3, 1, 1, 1, 0.6), PURE),
]


@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("jvp_mode", [1, 0])
@pytest.mark.parametrize("name,mesh,prm", SMALL_SYSTEMS, ids=[c[0] for c in SMALL_SYSTEMS])
def test_gmres_past_the_system_dimension(name, mesh, prm, jvp_mode, precond):
    """Systems of 16-18 unknowns with the 30-vector restart: the Krylov space fills the whole
    space within a cycle, where the new Arnoldi vector is rounding noise and ||w||^2 from the
    Pythagorean identity cancels to nothing (the residual estimate then ends the cycle). The
    steps must still converge to the direct-solve Newton solution (GMRES, Sec. 2.2)."""
    p = dataclasses.replace(prm, precond=precond, jvp_mode=jvp_mode, gmres_restart=30, gmres_maxit=300,
                            newton_rtol=1e-10)
    n = mesh.n_dofs
    Un = synth.seed_state(mesh, p, radius=0.5)
    Un = Un + 0.2 * synth.uniform_pm1(17, n)
    h = handle(mesh, p)
    dt = 0.1
    h.set_state(dev(Un), 0.0, dt)
    Uo, t, out = Un.copy(), 0.0, dev(np.zeros_like(Un))
    for _ in range(2):
        st = h.step()
        assert st["converged"] and st["fnorm"] < p.newton_rtol * st["fnorm0"], st
        Uo, ratio = OS.newton_direct(mesh, p, Uo, t, dt)
        assert ratio < 1e-12
        t += dt
        assert rel(host(h.get_state(out)), Uo) <= 1e-8


@pytest.mark.parametrize("name", ["alloy3d_256x256x128", "dendrite3d_192", "dendrite2d_1024"])
def test_full_size_residual_on_sampled_nodes(name):
    """At the full workload size the oracle evaluates sampled nodes one by one (Sec. 4.3 sizes)."""
    w = synth.workload(name)
    U0 = synth.initial_state(w)
    pert = 0.05 * synth.uniform_pm1(77, w.mesh.n_dofs)
    U = U0 + pert
    h = handle(w.mesh, dataclasses.replace(w.params, precond=0))
    h.set_state(dev(U0), 1.0, w.dt)
    F = host(h.residual(dev(U), dev(np.zeros_like(U))))
    n = w.mesh.n_nodes
    rng_nodes = (synth.splitmix64(5, 48) % np.uint64(n)).astype(np.int64)
    nodes = np.unique(np.concatenate([rng_nodes, [0, n - 1, w.mesh.nx, n // 2]]))
    rp, ru = OR.residual_at_nodes(w.mesh, w.params, U, U0, 1.0, w.dt, nodes)
    scale = max(np.abs(rp).max(), np.abs(ru).max())
    assert np.abs(F[nodes] - rp).max() <= 1e-12 * scale
    assert np.abs(F[n + nodes] - ru).max() <= 1e-12 * scale


@pytest.mark.parametrize("name", ["alloy3d_256x256x128", "dendrite3d_192", "dendrite2d_1024"])
def test_full_size_tangent_and_adjoint_on_sampled_nodes(name):
    """Exact J v (linearisation pass + tangent kernels, the launches of the timed step) and
    J^T w at the full workload size, against the oracle's complex-step products at sampled
    nodes (the directional derivative of Eqs. pf2/conc2, Sec. 2.2)."""
    w = synth.workload(name)
    U0 = synth.initial_state(w)
    U = U0 + 0.05 * synth.uniform_pm1(77, w.mesh.n_dofs)
    v = synth.uniform_pm1(78, w.mesh.n_dofs)
    wv = synth.uniform_pm1(79, w.mesh.n_dofs)
    prm = dataclasses.replace(w.params, precond=0, jvp_mode=1)
    h = handle(w.mesh, prm)
    h.set_state(dev(U0), 1.0, w.dt)
    tU, out = dev(U), dev(np.zeros_like(U))
    JV = host(h.jvp(tU, dev(v), out))
    JTW = host(h.jtvp(tU, dev(wv), out))
    n = w.mesh.n_nodes
    rng_nodes = (synth.splitmix64(6, 40) % np.uint64(n)).astype(np.int64)
    nodes = np.unique(np.concatenate([rng_nodes, [0, n - 1, w.mesh.nx, n // 2]]))
    jp, ju = OJ.jvp_at_nodes(w.mesh, prm, U, U0, 1.0, w.dt, v, nodes)
    scale = max(np.abs(jp).max(), np.abs(ju).max())
    assert np.abs(JV[nodes] - jp).max() <= 1e-12 * scale
    assert np.abs(JV[n + nodes] - ju).max() <= 1e-12 * scale
    tp, tu = OJ.jtvp_at_nodes(w.mesh, prm, U, U0, 1.0, w.dt, wv, nodes)
    scale = max(np.abs(tp).max(), np.abs(tu).max())
    assert np.abs(JTW[nodes] - tp).max() <= 1e-12 * scale
    assert np.abs(JTW[n + nodes] - tu).max() <= 1e-12 * scale


def test_error_codes():
    import paper_2006_16764_b300 as pkg

    mesh = Mesh(2, 8, 8, 0, 1.0)
    h = handle(mesh, PURE)
    U = dev(np.zeros(mesh.n_dofs))
    with pytest.raises(pkg.TusasError) as e:
        h.residual(U, dev(np.zeros(mesh.n_dofs)))
    assert e.value.code == pkg.EINVAL
    with pytest.raises(pkg.TusasError) as e:
        h.set_state(U, 0.0, -1.0)
    assert e.value.code == pkg.EINVAL
    with pytest.raises(pkg.TusasError) as e:
        pkg.Tusas(mesh, dataclasses.replace(PURE, k=0.5))
    assert e.value.code == pkg.EINVAL
    bad = synth.seed_state(mesh, PURE, 3.0)
    bad[5] = np.nan
    h.set_state(dev(bad), 0.0, 0.5)
    with pytest.raises(pkg.TusasError) as e:
        h.step()
    assert e.value.code == pkg.ENONFINITE
    h2 = handle(mesh, dataclasses.replace(PURE, newton_maxit=1))
    h2.set_state(dev(synth.seed_state(mesh, PURE, 3.0)), 0.0, 0.5)
    st = h2.step(allow_noconv=True)
    assert not st["converged"]
    with pytest.raises(pkg.TusasError) as e:
        h2.step()
    assert e.value.code == pkg.ENOCONV


def test_allocation_cap_gives_enomem_and_frees_everything():
    """A size cap makes the multigrid hierarchy (tusas_create) and the linearisation store
    (first exact-tangent step) fail with TUSAS_ENOMEM; nothing stays allocated."""
    import paper_2006_16764_b300 as pkg

    import gc

    gc.collect()  # handles of earlier tests that are no longer referenced
    mesh = Mesh(3, 16, 16, 16, 1.0)
    base = 8 * mesh.n_dofs * (11 + 2 * 30 + 1) + 8 * (592 * 32 + 256)
    held = pkg.device_bytes()
    try:
        pkg.set_device_bytes_cap(held + base + 4096)
        with pytest.raises(pkg.TusasError) as e:
            pkg.Tusas(mesh, Params(model=0, precond=2, jvp_mode=1))
        assert e.value.code == pkg.ENOMEM
        assert pkg.device_bytes() == held
        pkg.set_device_bytes_cap(0)
        h = pkg.Tusas(mesh, Params(model=0, precond=1, jvp_mode=1))
        pkg.set_device_bytes_cap(pkg.device_bytes() + 1024)
        h.set_state(dev(synth.seed_state(mesh, PURE, 3.0)), 0.0, 0.5)
        with pytest.raises(pkg.TusasError) as e:
            h.step()
        assert e.value.code == pkg.ENOMEM
        pkg.set_device_bytes_cap(0)
        assert h.step()["converged"]
        h.close()
        assert pkg.device_bytes() == held
    finally:
        pkg.set_device_bytes_cap(0)


def test_dendrite2d_128_ten_steps_match_oracle():
    """The 128^2 pure-metal workload, all 10 backward-Euler steps (FD-JFNK, point Jacobi)."""
    w = synth.workload("dendrite2d_128")
    U0 = synth.initial_state(w)
    h = handle(w.mesh, w.params)
    h.set_state(dev(U0), 0.0, w.dt)
    Uo, t = U0.copy(), 0.0
    out = dev(np.zeros_like(U0))
    for _ in range(w.steps):
        st = h.step()
        assert st["converged"]
        Uo, ratio = OS.newton_direct(w.mesh, w.params, Uo, t, w.dt)
        assert ratio < 1e-12
        t += w.dt
    assert rel(host(h.get_state(out)), Uo) <= 1e-8


THETA_CASES = [
    ("2d-pure-cn", Mesh(2, 21, 13, 0, 0.9), dataclasses.replace(PURE, theta=0.5, phihat_form=1)),
    ("2d-alloy-cn-eqtheta", Mesh(2, 19, 11, 0, 0.8), dataclasses.replace(ALLOY, theta=0.5, phihat_form=0)),
    ("3d-alloy-theta0.7", Mesh(3, 9, 6, 7, 0.8), dataclasses.replace(ALLOY, theta=0.7, phihat_form=0)),
    ("3d-pure-cn-literal", Mesh(3, 7, 5, 6, 0.9), dataclasses.replace(PURE, theta=0.5, phihat_form=1, time_form=1)),
]


@pytest.mark.parametrize("name,mesh,prm", THETA_CASES, ids=[c[0] for c in THETA_CASES])
def test_theta_method_residual_tangent_adjoint(name, mesh, prm):
    """theta-method (Eqs. dpf, dc, theta): level-n spatial terms, U^{n-1} history, tangent and J^T."""
    import paper_2006_16764_b300 as pkg

    U, Un = _inputs(mesh, 13)
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
    if prm.phihat_form == 1:
        # level-n spatial terms weighted (1 - theta) in (dF/dU^n)^T w and dF/d eps4
        h.jtvp_prev(tU, dev(w), out)
        assert rel(host(out), OJ.dF_dUn_T(mesh, prm, U, Un, tn, dt, w)) <= 1e-12
        h.dFdp(tU, out, 0)
        assert rel(host(out), OJ.dF_deps4(mesh, prm, U, Un, tn, dt)) <= 1e-12
    else:
        with pytest.raises(pkg.TusasError):
            h.dFdp(tU, out, 0)


@pytest.mark.parametrize("form", [1, 0])
def test_crank_nicolson_steps_match_oracle(form):
    w = synth.scaled(synth.workload("dendrite2d_1024"), 32, 32)
    prm = dataclasses.replace(w.params, theta=0.5, phihat_form=form, jvp_mode=1, precond=2)
    U0 = synth.initial_state(w)
    h = handle(w.mesh, prm)
    h.set_state(dev(U0), 0.0, w.dt)
    Uo, Uprev, t = U0.copy(), U0.copy(), 0.0
    out = dev(np.zeros_like(U0))
    for _ in range(3):
        st = h.step()
        assert st["converged"]
        Unew, ratio = OS.newton_direct(w.mesh, prm, Uo, t, w.dt, Unm1=Uprev)
        assert ratio < 1e-12
        Uprev, Uo = Uo, Unew
        t += w.dt
        assert rel(host(h.get_state(out)), Uo) <= 1e-8
