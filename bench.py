#!/usr/bin/env python
"""Benchmark of the B300 hot path on the 3D dilute-alloy phase-field problem
(256x256x128 Q1 hexes, 17,040,642 dofs).

The timed steps are backward-Euler Newton-Krylov time steps through the whole
hot path: residual F(U), pointwise linearisation, exact tangent J v, FP32
block-Jacobi / GMG preconditioner fill and apply, FGMRES(30) with CGS2,
Newton update and line search (`ms_per_step`). The headline `value` is the
metric's residual rate: isolated evaluations of F over all dofs per second
(CUDA events, `steps` evaluations of the converged state). The same line
reports the dominant kernel's roofline (FP64 pipe, and HBM against the
nodal bytes), exact tangent + FP32 multigrid against FD J v + FP64 multigrid
over the same steps (at the workload's GMRES cap and at 30), end-to-end
numbers through the C-ABI with host buffers, and the CPU oracle on a bounded
sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "3D residual Mdof-evals/s (%HBM roofline); JFNK s/step exact-JVP+FP32 vs FD-FP64"
UNIT = "Mdof-evals/s"
WORKLOAD = "alloy3d_256x256x128"
# Oracle sample for the CPU baseline: the same physics, spacing, time step and
# initial front on a 48x48x32 sub-box (about 150k dofs per evaluation).
CPU_SAMPLE = (48, 48, 32)

# FP64-pipe lane slots per element of one element-tile pass (ncu sm__inst_executed_pipe_fp64.sum
# x 32 over its 8 colour launches / elements, a one-pass counter): the arithmetic, the compares,
# the conversions and the inactive lanes of every FP64 instruction. Measured on the full
# 256x256x128 alloy box in the state the bench times: the isolated residual on the converged
# state (its flat Gauss points skip the anisotropy), the mean of the 5 linearisation passes of
# one step (1297-1378), the tangent (its instruction stream does not depend on the data).
# Against the pipe's slot rate (the FMA-chain peak / 2) they give its occupancy.
FP64_PIPE_SLOTS_PER_ELEM = {"residual": 739.5, "residual_lin": 1336.2, "jv": 501.0}
# On the 256x192x64 profiling box, per element: the same slots, and the FP64 flops of the
# compiled kernels (DADD + DMUL + 2 DFMA: smsp__sass_thread_inst_executed_op_d{add,mul,fma}_pred_on,
# which take three passes and so are not captured on the full box).
PROFILE_PIPE_SLOTS_PER_ELEM = {"residual": 827.5, "residual_lin": 1388.5, "jv": 501.0}
PROFILE_FLOPS_PER_ELEM = {"residual": 1149.3, "residual_lin": 1891.3, "jv": 802.7}
# FP64 flops per element on the full box: its slots times the profiling box's flops per slot
# (exact for the tangent; an estimate for the residual passes, whose skipped work has about
# the mix of the rest).
FP64_FLOPS_PER_ELEM = {k: FP64_PIPE_SLOTS_PER_ELEM[k] * PROFILE_FLOPS_PER_ELEM[k] / PROFILE_PIPE_SLOTS_PER_ELEM[k]
                       for k in FP64_PIPE_SLOTS_PER_ELEM}
# Algorithmic HBM bytes per node of the method's operators: F reads U, U^n and
# writes F (6 doubles); J v also reads v (8 doubles). Coordinates are implicit.
ALG_BYTES_PER_NODE = {"residual": 48.0, "residual_lin": 48.0, "jv": 64.0}
# The stored pointwise linearisation (22 coefficients x 8 Gauss points per
# element) is this implementation's trade of HBM traffic for FP64 work; it is
# reported beside the roofline, not counted as algorithmic bytes.
LIN_BYTES_PER_ELEM = 22 * 8 * 8.0
# DRAM bytes per element measured by ncu on the same pass (dram__bytes_read.sum +
# dram__bytes_write.sum over the 8 colour launches / elements); the traffic scales
# with the elements processed (same tiles, same per-element streams).
NCU_BYTES_PER_ELEM = {"residual": 153.2, "residual_lin": 1447.7, "jv": 1544.7}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fd-steps", type=int, default=5,
                    help="FD-JFNK + FP64 steps from the same start state as the first timed steps")
    ap.add_argument("--cap30-steps", type=int, default=3,
                    help="steps of both arms with one full GMRES(30) cycle per Newton iteration")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--e2e-evals", type=int, default=20,
                    help="residual evaluations streamed through the end-to-end measurement (host U in, "
                         "F out); the first copy in and the last copy out are the pipeline's fill and drain")
    ap.add_argument("--cpu-seconds", type=float, default=18.0)
    ap.add_argument("--report", default=None, choices=synth.WORKLOADS + ["q2", "q2hex"],
                    help="run one workload's full protocol (step counts, precision / tangent comparisons, "
                         "adjoint gradients) and print a JSON summary; q2: biquadratic vs Q1 elements on "
                         "the dendrite2d_1024 box; q2hex: triquadratic vs Q1 hexes on the dendrite3d_192 box")
    ap.add_argument("--kernels", nargs="?", const="alloy3d", default=None, choices=["alloy3d", "q2", "pc", "gmres"],
                    help="profiling case: a few residual / linearisation / tangent passes on a 256x192x64 "
                         "sub-box of the alloy workload (inputs > L2, about 5 GB on the device), or (q2) on "
                         "a 1536^2 Q2 box of the 2D dendrite (about 2 GB), or (pc) 2 preconditioner setups and "
                         "3 applies (FP32 GMG) on the same alloy sub-box, or (gmres) one FD-JFNK step there")
    return ap.parse_args()


def run_kernels(kind="alloy3d"):
    """Small case for detailed counters: 2 residuals, then 2 tangent actions (each a
    linearisation pass and a tangent pass); every pass is one launch per tile colour."""
    import dataclasses

    import torch

    import paper_2006_16764_b300 as pkg

    if kind == "gmres":
        # one FD-JFNK step with the FP32 multigrid (no linearisation store: about 4 GB on the device)
        w = synth.scaled(synth.workload(WORKLOAD), 256, 192, 64)
        prm = dataclasses.replace(w.params, jvp_mode=0, smoother_fp32=1)
        dev = torch.device("cuda", 0)
        h = pkg.Tusas(w.mesh, prm)
        h.set_state(torch.tensor(synth.initial_state(w), device=dev), 0.0, w.dt)
        st = h.step()
        torch.cuda.synchronize()
        print(json.dumps({"kernels": kind, "dofs": w.mesh.n_dofs, "gmres_its": st["gmres_its"]}))
        h.close()
        return
    if kind == "pc":
        w = synth.scaled(synth.workload(WORKLOAD), 256, 192, 64)
        dev = torch.device("cuda", 0)
        U0 = torch.tensor(synth.initial_state(w), device=dev)
        U = U0 + 0.01 * torch.tensor(synth.uniform_pm1(3, w.mesh.n_dofs), device=dev)
        r = torch.tensor(synth.uniform_pm1(4, w.mesh.n_dofs), device=dev)
        h = pkg.Tusas(w.mesh, w.params)
        h.set_state(U0, 0.0, w.dt)
        z = torch.empty_like(r)
        for _ in range(2):
            h.precond_setup(U)
        for _ in range(3):
            h.precond_apply(r, z)
        torch.cuda.synchronize()
        print(json.dumps({"kernels": kind, "dofs": w.mesh.n_dofs, "elems": w.mesh.n_elems}))
        h.close()
        return
    if kind == "q2":
        base = synth.workload("dendrite2d_1024")
        mesh = synth.Mesh(2, 1536, 1536, 0, 400.0 / 1536, order=2)
        w = synth.Workload("dendrite2d_q2_1536", mesh, base.params, base.dt, 1)
        U0h = synth.seed_state(mesh, base.params, radius=8.0)
    else:
        w = synth.scaled(synth.workload(WORKLOAD), 256, 192, 64)
        U0h = synth.initial_state(w)
    prm = dataclasses.replace(w.params, gmres_restart=2, precond=0)
    dev = torch.device("cuda", 0)
    U0 = torch.tensor(U0h, device=dev)
    U = U0 + 0.01 * torch.tensor(synth.uniform_pm1(3, w.mesh.n_dofs), device=dev)
    v = torch.tensor(synth.uniform_pm1(4, w.mesh.n_dofs), device=dev)
    h = pkg.Tusas(w.mesh, prm)
    h.set_state(U0, 0.0, w.dt)
    F = torch.empty_like(U)
    for _ in range(2):
        h.residual(U, F)
    for _ in range(2):
        h.jvp(U, v, F)
    torch.cuda.synchronize()
    print(json.dumps({"kernels": kind, "dofs": w.mesh.n_dofs, "elems": w.mesh.n_elems}))
    h.close()


# ----------------------------------------------------------------------------
def _timed_steps(h, n, stream):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = [h.step() for _ in range(n)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, st


def _run_variant(w, prm, U0, nsteps, stream):
    """nsteps implicit steps; stops at the first step that does not converge and says so."""
    import torch

    import paper_2006_16764_b300 as pkg

    h = pkg.Tusas(w.mesh, prm, stream=stream)
    h.set_state(U0, 0.0, w.dt)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = []
    failed = None
    for i in range(nsteps):
        s = h.step(allow_noconv=True)
        st.append(s)
        if not s["converged"]:
            failed = i + 1
            break
    e1.record(stream)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    U = torch.empty_like(U0)
    h.get_state(U)
    h.close()
    return {"s_per_step": secs / len(st), "steps_done": len(st), "newton_its": [s["newton_its"] for s in st],
            "gmres_its": [s["gmres_its"] for s in st], "converged": failed is None,
            "first_failed_step": failed}, U


def _operator_rates(mesh, prm, stream, reps=20):
    """ms per residual, linearisation (residual + stored pointwise Jacobian) and tangent pass."""
    import dataclasses

    import torch

    import paper_2006_16764_b300 as pkg

    dev = torch.device("cuda", 0)
    h = pkg.Tusas(mesh, dataclasses.replace(prm, precond=0, gmres_restart=1), stream=stream)
    U0 = torch.tensor(synth.seed_state(mesh, prm, radius=8.0), device=dev)
    U = U0 + 0.01 * torch.tensor(synth.uniform_pm1(3, mesh.n_dofs), device=dev)
    v = torch.tensor(synth.uniform_pm1(4, mesh.n_dofs), device=dev)
    h.set_state(U0, 0.0, 0.5)
    F = torch.empty_like(U)
    for _ in range(3):
        h.residual(U, F)
        h.jvp(U, v, F)
    h.timers(True)
    for _ in range(reps):
        h.residual(U, F)
        h.jvp(U, v, F)
    t = h.get_timers()
    h.timers(False)
    h.close()
    out = {"dofs": mesh.n_dofs, "elems": mesh.n_elems}
    for k in ("residual", "residual_lin", "jv"):
        ms = t[k][0] / max(t[k][1], 1)
        out[k] = {"ms": ms, "Mdof_evals_per_s": mesh.n_dofs / ms / 1e3}
    return out


def run_q2_report(stream):
    """Biquadratic (Q2, 3x3 Gauss) against Q1 elements on the 400 x 400 box of the 2D dendrite.

    Kernel rates at equal node counts (Q2 with n elements per axis vs Q1 with 2n), and
    backward-Euler JFNK steps of the dendrite seed with the same node spacing:
    Q2 512^2 (point Jacobi, and multigrid from the h/2 node lattice) against Q1 1024^2
    with point Jacobi and with the GMG V-cycle.
    """
    import dataclasses

    import torch

    w = synth.workload("dendrite2d_1024")
    out = {"report": "q2"}
    rates = []
    for n in (256, 512, 1024, 2048):
        m2 = synth.Mesh(2, n, n, 0, 400.0 / n, order=2)
        m1 = synth.Mesh(2, 2 * n, 2 * n, 0, 200.0 / n)
        rates.append({"q2_elems_per_axis": n, "q2": _operator_rates(m2, w.params, stream),
                      "q1_same_nodes": _operator_rates(m1, w.params, stream)})
    out["operator_rates"] = rates
    dev = torch.device("cuda", 0)
    nsteps = 10
    m2 = synth.Mesh(2, 512, 512, 0, 400.0 / 512, order=2)
    variants = [("q2_512_exact_jacobi", m2, dict(precond=1, jvp_mode=1)),
                ("q2_512_fd_jacobi", m2, dict(precond=1, jvp_mode=0)),
                ("q2_512_exact_gmg_fp32", m2, dict(precond=2, jvp_mode=1, smoother_fp32=1, cheb_degree=3)),
                ("q1_1024_exact_jacobi", w.mesh, dict(precond=1, jvp_mode=1)),
                ("q1_1024_exact_gmg_fp32", w.mesh, dict(precond=2, jvp_mode=1, smoother_fp32=1))]
    for name, mesh, opts in variants:
        prm = dataclasses.replace(w.params, newton_maxit=30, **opts)
        U0 = torch.tensor(synth.seed_state(mesh, prm, radius=8.0), device=dev)
        ws = synth.Workload(name, mesh, prm, w.dt, nsteps)
        r, _ = _run_variant(ws, prm, U0, nsteps, stream)
        out[name] = r
    print(json.dumps(out), flush=True)


def run_q2hex_report(stream):
    """Triquadratic (Q2 hex, 3x3x3 Gauss) against trilinear (Q1) elements in 3D.

    Kernel rates at equal node counts (Q2 with n elements per axis against Q1 with 2n) on the
    [-76.8, 76.8]^3 box of the 3D dendrite, and backward-Euler Newton-Krylov steps of its
    centred seed at the same node spacing (0.8): Q2 48^3 with point Jacobi and with the FP32
    multigrid from its node lattice, against Q1 96^3 with point Jacobi and with the FP32
    multigrid V-cycle.
    """
    import dataclasses

    import torch

    w = synth.workload("dendrite3d_192")
    out = {"report": "q2hex"}
    rates = []
    for n in (32, 64, 96):
        hq = 153.6 / n
        m2 = synth.Mesh(3, n, n, n, hq, -76.8, -76.8, -76.8, order=2)
        m1 = synth.Mesh(3, 2 * n, 2 * n, 2 * n, hq / 2, -76.8, -76.8, -76.8)
        rates.append({"q2_elems_per_axis": n, "q2": _operator_rates(m2, w.params, stream),
                      "q1_same_nodes": _operator_rates(m1, w.params, stream)})
    out["operator_rates"] = rates
    dev = torch.device("cuda", 0)
    nsteps = 5
    m2 = synth.Mesh(3, 48, 48, 48, 1.6, -38.4, -38.4, -38.4, order=2)
    m1 = synth.Mesh(3, 96, 96, 96, 0.8, -38.4, -38.4, -38.4)
    variants = [("q2hex_48_exact_jacobi", m2, dict(precond=1, jvp_mode=1)),
                ("q1_96_exact_jacobi", m1, dict(precond=1, jvp_mode=1)),
                ("q2hex_48_exact_gmg_fp32", m2, dict(precond=2, jvp_mode=1, smoother_fp32=1, cheb_degree=3)),
                ("q1_96_exact_gmg_fp32", m1, dict(precond=2, jvp_mode=1, smoother_fp32=1))]
    sols = {}
    for name, mesh, opts in variants:
        prm = dataclasses.replace(w.params, newton_maxit=30, gmres_maxit=300, **opts)
        U0 = torch.tensor(synth.seed_state(mesh, prm, radius=10.0, centred=True), device=dev)
        ws = synth.Workload(name, mesh, prm, w.dt, nsteps)
        r, U = _run_variant(ws, prm, U0, nsteps, stream)
        out[name] = r
        sols[name] = U
    # solid fraction of the two discretisations after the same steps (the accuracy lever of Sec. 4.1)
    import paper_2006_16764_b300 as pkg

    for name, mesh, opts in variants[:2]:
        h = pkg.Tusas(mesh, dataclasses.replace(w.params, precond=0), stream=stream)
        out[name]["solid_fraction"] = h.solid_fraction(sols[name])
        h.close()
    print(json.dumps(out), flush=True)


def run_report(name):
    """Each workload's protocol: step counts, tangent / precision comparisons, adjoint gradients."""
    import dataclasses

    import torch

    import paper_2006_16764_b300 as pkg

    if name == "q2":
        return run_q2_report(torch.cuda.current_stream(torch.device("cuda", 0)))
    if name == "q2hex":
        return run_q2hex_report(torch.cuda.current_stream(torch.device("cuda", 0)))
    w = synth.workload(name)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    U0 = torch.tensor(synth.initial_state(w), device=dev)
    out = {"report": name, "dofs": w.mesh.n_dofs, "dt": w.dt, "steps": w.steps,
           "kappa": 2 * w.dt * (w.params.D / (1 + w.params.k)) / w.mesh.h ** 2}
    if name == "dendrite2d_128":
        r, U = _run_variant(w, w.params, U0, w.steps, stream)
        out["fd_jfnk_jacobi_fp64"] = r
        Ur, Un = synth.random_fields(w.mesh, 42)
        h = pkg.Tusas(w.mesh, w.params, stream=stream)
        h.set_state(torch.tensor(Un, device=dev), 0.0, w.dt)
        tU = torch.tensor(Ur, device=dev)
        F = torch.empty_like(tU)
        h.residual(tU, F)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(100):
            h.residual(tU, F)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 100
        out["residual_100_evals"] = {"ms_per_eval": ms, "Mdof_evals_per_s": w.mesh.n_dofs / ms / 1e3}
        h.close()
        # the CPU oracle on one host core: the same residual and the first backward-Euler step
        from oracle import residual as OR
        from oracle import solver as OS

        t0 = time.perf_counter()
        OR.residual(w.mesh, w.params, Ur, Un, 0.0, w.dt)
        t1 = time.perf_counter()
        Uo, so = OS.newton_step(w.mesh, w.params, synth.initial_state(w), 0.0, w.dt)
        t2 = time.perf_counter()
        out["oracle_1core"] = {"residual_s": t1 - t0, "first_step_s": t2 - t1, "newton_its": so.newton_its,
                               "gmres_its": so.gmres_its, "converged": so.converged,
                               "gpu_s_per_step_mean": r["s_per_step"]}
    elif name == "dendrite2d_1024":
        sweep = []
        for n in (128, 256, 512, 1024, 2048, 4096):
            ws = synth.scaled(w, n, n)
            ws.mesh.h = 400.0 / n
            h = pkg.Tusas(ws.mesh, dataclasses.replace(w.params, precond=0, gmres_restart=1), stream=stream)
            Us = torch.tensor(synth.initial_state(ws), device=dev)
            h.set_state(Us, 0.0, w.dt)
            F = torch.empty_like(Us)
            for _ in range(3):
                h.residual(Us, F)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = 20
            e0.record(stream)
            for _ in range(reps):
                h.residual(Us, F)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            sweep.append({"n": n, "dofs": ws.mesh.n_dofs, "ms": ms, "Mdof_evals_per_s": ws.mesh.n_dofs / ms / 1e3})
            h.close()
            del Us, F
        out["residual_sweep"] = sweep
        from oracle import residual as OR

        Uh = synth.initial_state(w)
        t0 = time.perf_counter()
        OR.residual(w.mesh, w.params, Uh, Uh, 0.0, w.dt)
        out["oracle_1core_residual_s"] = time.perf_counter() - t0
        base = dataclasses.replace(w.params, newton_maxit=30)
        r32, U32 = _run_variant(w, dataclasses.replace(base, smoother_fp32=1), U0, w.steps, stream)
        r64, U64 = _run_variant(w, dataclasses.replace(base, smoother_fp32=0), U0, w.steps, stream)
        rex, Uex = _run_variant(w, dataclasses.replace(base, smoother_fp32=1, jvp_mode=1), U0, w.steps, stream)
        out["fd_jfnk_gmg_fp32"] = r32
        out["fd_jfnk_gmg_fp64"] = r64
        out["exact_jfnk_gmg_fp32"] = rex
        out["fp32_vs_fp64_solution_rel_inf"] = float((U32 - U64).abs().max() / U64.abs().max())
    elif name == "dendrite3d_192":
        r32, U32 = _run_variant(w, dataclasses.replace(w.params, smoother_fp32=1), U0, w.steps, stream)
        r64, U64 = _run_variant(w, dataclasses.replace(w.params, smoother_fp32=0), U0, w.steps, stream)
        out["exact_jfnk_gmg_fp32"] = r32
        out["exact_jfnk_gmg_fp64"] = r64
        out["fp32_vs_fp64_solution_rel_inf"] = float((U32 - U64).abs().max() / U64.abs().max())
    elif name == "alloy3d_256x256x128":
        rex, Uex = _run_variant(w, dataclasses.replace(w.params, jvp_mode=1, smoother_fp32=1), U0, w.steps, stream)
        rfd, Ufd = _run_variant(w, dataclasses.replace(w.params, jvp_mode=0, smoother_fp32=1), U0, w.steps, stream)
        rfd64, Ufd64 = _run_variant(w, dataclasses.replace(w.params, jvp_mode=0, smoother_fp32=0), U0, w.steps, stream)
        out["exact_jv_gmg_fp32"] = rex
        out["fd_jv_gmg_fp32"] = rfd
        out["fd_jv_gmg_fp64"] = rfd64
        out["exact_vs_fd_solution_rel_inf"] = float((Uex - Ufd).abs().max() / Ufd.abs().max())
        out["exact_fp32_vs_fd_fp64_solution_rel_inf"] = float((Uex - Ufd64).abs().max() / Ufd64.abs().max())
    elif name == "adjoint2d_512":
        from paper_2006_16764_b300.adjoint import SolidFraction, SolidFractionProblem

        nn = w.mesh.n_nodes
        # tight Newton tolerance for the finite-difference check (1e-13 and 1e-12 are at the
        # FP64 roundoff floor of ||F|| at this size: ||F||/||F0|| stalls near 5e-13 on some steps)
        prm = dataclasses.replace(w.params, jvp_mode=1, newton_rtol=1e-11)
        h = pkg.Tusas(w.mesh, prm, stream=stream)
        pb = SolidFractionProblem(
            h, prm, lambda d: torch.tensor(synth.initial_state(
                synth.Workload(w.name, w.mesh, dataclasses.replace(prm, Delta=d), w.dt, w.steps)), device=dev),
            torch.tensor(np.concatenate([np.zeros(nn), -np.ones(nn)]), device=dev),
            0.0, w.dt, w.steps, 10, 1e-12)
        r = synth.uniform01(3, 16)
        samples = []
        for i in range(8):
            e4 = 0.02 + 0.04 * r[2 * i]
            dl = 0.45 + 0.30 * r[2 * i + 1]
            te = torch.tensor(e4, dtype=torch.float64, requires_grad=True)
            td = torch.tensor(dl, dtype=torch.float64, requires_grad=True)
            h.timers(True)
            t0 = time.perf_counter()
            S = SolidFraction.apply(te, td, pb)
            t1 = time.perf_counter()
            ge, gd = torch.autograd.grad(S, (te, td))
            t2 = time.perf_counter()
            tm = h.get_timers()
            h.timers(False)
            samples.append({"eps4": e4, "Delta": dl, "S": float(S), "dS_deps4": float(ge), "dS_dDelta": float(gd),
                            "forward_s": t1 - t0, "adjoint_s": t2 - t1,
                            "forward_gmres": pb.last_forward["gmres_its"], "adjoint_gmres": pb.last_adjoint["gmres_its"],
                            # device time of the operator classes (CUDA events around each application)
                            "operator_device_s": sum(v[0] for v in tm.values()) / 1e3})
        out["samples"] = samples
        # the same 8 samples at once: 8 handles on 8 streams, one host thread each
        from paper_2006_16764_b300.adjoint import solid_fraction_batch

        probs = []
        for _ in samples:
            s_ = torch.cuda.Stream(dev)
            probs.append(SolidFractionProblem(
                pkg.Tusas(w.mesh, prm, stream=s_), prm, pb.initial_state, pb.dU0_ddelta, 0.0, w.dt,
                w.steps, 10, 1e-12, stream=s_))
        sam = [(x["eps4"], x["Delta"]) for x in samples]
        solid_fraction_batch(probs[:1], sam[:1])  # allocate the first handle's checkpoints outside the timing
        util = UtilSampler(0)
        util.start()
        t0 = time.perf_counter()
        res = solid_fraction_batch(probs, sam)
        t1 = time.perf_counter()
        out["batch_gpu_utilization"] = util.stop()
        out["batch_of_8"] = {
            "seconds": t1 - t0,
            "sequential_seconds": sum(x["forward_s"] + x["adjoint_s"] for x in samples),
            "max_abs_diff_vs_sequential": max(
                max(abs(r_["S"] - x["S"]), abs(r_["dS_deps4"] - x["dS_deps4"]), abs(r_["dS_dDelta"] - x["dS_dDelta"]))
                for r_, x in zip(res, samples))}
        for p_ in probs:
            p_.handle.close()
        # central differences (h = 1e-6) for the first sample, Newton tolerance 1e-13
        hh = 1e-6
        s0 = samples[0]
        out["newton_rtol"] = prm.newton_rtol

        def S_at(e4, dl):
            return float(SolidFraction.apply(torch.tensor(e4, dtype=torch.float64), torch.tensor(dl, dtype=torch.float64), pb))

        fd_e = (S_at(s0["eps4"] + hh, s0["Delta"]) - S_at(s0["eps4"] - hh, s0["Delta"])) / (2 * hh)
        fd_d = (S_at(s0["eps4"], s0["Delta"] + hh) - S_at(s0["eps4"], s0["Delta"] - hh)) / (2 * hh)
        out["fd_check"] = {"h": hh, "dS_deps4_fd": fd_e, "dS_dDelta_fd": fd_d,
                           "rel_err_eps4": abs(s0["dS_deps4"] - fd_e) / abs(fd_e),
                           "rel_err_Delta": abs(s0["dS_dDelta"] - fd_d) / abs(fd_d)}
        h.close()
    print(json.dumps(out), flush=True)


def cpu_oracle_rate(seconds, warm=0):
    """Oracle residual evaluations on the bounded sample on 1 host core: the median of the
    per-evaluation times over about `seconds`, as Mdof-evals/s."""
    from oracle import residual as OR

    w = synth.scaled(synth.workload(WORKLOAD), *CPU_SAMPLE)
    U0 = synth.initial_state(w)
    U = U0 + 0.01 * synth.uniform_pm1(5, w.mesh.n_dofs)
    for _ in range(warm):
        OR.residual(w.mesh, w.params, U, U0, 0.0, w.dt)
    per = []
    t0 = time.perf_counter()
    while True:
        t1 = time.perf_counter()
        OR.residual(w.mesh, w.params, U, U0, 0.0, w.dt)
        per.append(time.perf_counter() - t1)
        if time.perf_counter() - t0 >= seconds:
            break
    return w.mesh.n_dofs / statistics.median(per) / 1e6, len(per), sum(per), w


# ---- the oracle on all host cores: element chunks in spawned worker processes ----------
_POOL_STATE = {}


def _pool_init(root):
    if root not in sys.path:
        sys.path.insert(0, root)
    w = synth.scaled(synth.workload(WORKLOAD), *CPU_SAMPLE)
    U0 = synth.initial_state(w)
    _POOL_STATE.update(w=w, U0=U0, U=U0 + 0.01 * synth.uniform_pm1(5, w.mesh.n_dofs))


def _pool_chunk(rng):
    """Residual contributions of elements [s, e) of the sample (oracle functions, as in its own loop)."""
    from oracle import fem
    from oracle import residual as OR

    st = _POOL_STATE
    w, U, U0 = st["w"], st["U"], st["U0"]
    mesh, n = w.mesh, w.mesh.n_nodes
    elems = fem.all_elements(mesh)[:, rng[0]:rng[1]]
    conn = fem.connectivity(mesh, elems)
    phi_e, u_e = OR.gather(mesh, U, conn)
    phin_e, un_e = OR.gather(mesh, U0, conn)
    c = OR.element_residual(mesh, w.params, elems, phi_e, u_e, phin_e, un_e, 0.0, w.dt, None, None)
    return np.concatenate([fem.scatter_add(n, conn, c[:, 0, :]), fem.scatter_add(n, conn, c[:, 1, :])])


class OraclePool:
    """The oracle residual of the bounded sample split over `procs` spawned processes (element
    chunks, partial vectors summed in chunk order): the oracle as it stands on all host cores."""

    def __init__(self, procs=None):
        import multiprocessing as mp

        self.procs = procs or min(os.cpu_count() or 1, 64)
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_pool_init, initargs=(ROOT,))
        w = synth.scaled(synth.workload(WORKLOAD), *CPU_SAMPLE)
        self.w = w
        E = w.mesh.n_elems
        cuts = [E * i // self.procs for i in range(self.procs + 1)]
        self.ranges = [(cuts[i], cuts[i + 1]) for i in range(self.procs)]

    def evaluate(self):
        parts = self.pool.map_async(_pool_chunk, self.ranges).get(timeout=600)
        F = parts[0].copy()
        for p in parts[1:]:
            F += p
        return F

    def rate(self, seconds, warm=2):
        """Mdof-evals/s from the median per-evaluation time over about `seconds` (the host is
        shared, so a median is steadier than a mean); also the evaluations and their spread."""
        for _ in range(warm):
            self.evaluate()
        per = []
        t0 = time.perf_counter()
        while True:
            t1 = time.perf_counter()
            self.evaluate()
            per.append(time.perf_counter() - t1)
            if time.perf_counter() - t0 >= seconds:
                break
        per.sort()
        q = lambda f: per[min(len(per) - 1, int(f * len(per)))]  # noqa: E731
        return (self.w.mesh.n_dofs / statistics.median(per) / 1e6, len(per), sum(per),
                {"min_s": per[0], "median_s": statistics.median(per), "p90_s": q(0.9)})

    def close(self):
        self.pool.close()
        self.pool.join()


class UtilSampler:
    """nvidia-smi utilization.gpu (percent of the sample period with a kernel running) every 100 ms."""

    def __init__(self, index):
        self.rows = []
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=utilization.gpu",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=lambda: self.rows.extend(line.strip() for line in self.proc.stdout),
                                       daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        v = [float(r) for r in self.rows if r.replace(".", "").isdigit()]
        return {"samples": len(v), "mean_pct": statistics.mean(v) if v else None,
                "median_pct": statistics.median(v) if v else None}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.rows = []
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        import torch

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(ws, x, dev):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(ws, x, dev):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------
def bench_config(w, ws):
    """The `config` object of both arms (the workload, its solver controls, L2 policy)."""
    prm, mesh = w.params, w.mesh
    return {"workload": w.name, "mesh": f"{mesh.nx}x{mesh.ny}x{mesh.nz} Q1 hex, h={mesh.h}", "dofs": mesh.n_dofs,
            "dt": w.dt, "jvp": "exact (stored pointwise linearisation)",
            "precond": f"block Jacobi, GMG V-cycle ({prm.mg_levels} levels), Chebyshev({prm.cheb_degree}), "
                       f"{'FP32' if prm.smoother_fp32 else 'FP64'}",
            "newton_rtol": prm.newton_rtol, "gmres_restart": prm.gmres_restart,
            "gmres_maxit_per_newton": prm.gmres_maxit,
            "l2": f"inputs larger than L2 (state {8 * mesh.n_dofs / 1e6:.0f} MB per vector, linearisation "
                  f"{LIN_BYTES_PER_ELEM * mesh.n_elems / 1e9:.1f} GB), no flush",
            "parallelism": f"{ws} independent replica(s)"}


VALUE_DEF = ("value: isolated residual F(U) (tusas_residual, Eqs. pf2/conc2 with the 2x2x2 Gauss rule) "
             "over all dofs, evaluations x dofs / s, CUDA events over `steps` back-to-back evaluations "
             "of a converged alloy state; ms_per_step: one backward-Euler Newton-Krylov time step "
             "(exact tangent, FP32 multigrid), the timed region of `steps` steps")


def run_reference(args, ws, rank):
    """The CPU oracle as it stands, on rank 0 only: residual evaluations on the bounded sample."""
    if rank != 0:
        return
    pool = OraclePool()
    pool.evaluate()
    w = pool.w
    per = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pool.evaluate()
        if i >= args.warmup:
            per.append(time.perf_counter() - t0)
    pool.close()
    secs = sum(per)
    # median per-evaluation time: the host is shared, a median is steadier than the mean
    value = w.mesh.n_dofs / statistics.median(per) / 1e6
    sample = (f"oracle residual on the {CPU_SAMPLE[0]}x{CPU_SAMPLE[1]}x{CPU_SAMPLE[2]} sub-box of {WORKLOAD} "
              f"({w.mesh.n_dofs} dofs), one evaluation per step (median of {len(per)}), element chunks over "
              f"{pool.procs} processes")
    full = synth.workload(WORKLOAD)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(full, args.gpus), "value_def": "oracle residual rate on the sample (Mdof-evals/s)",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _hbm_peak():
    """HBM copy bandwidth (GB/s) written by the GPU-pool driver, else the profiling fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback 6.4 TB/s (no MEASURED_PEAKS.json)"


def _steps_timed(h, n, stream):
    """n Newton-Krylov steps with one CUDA-event pair per step on `stream`: (seconds per step, stats)."""
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    st = []
    ev[0].record(stream)
    for i in range(n):
        st.append(h.step(allow_noconv=True))
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) / 1e3 for i in range(n)], st


def _arm(pkg, mesh, prm, Ustart, t_start, dt, n, stream):
    """n steps of one solver variant from (Ustart, t_start): per-step seconds, Newton/GMRES counts, timers."""
    h = pkg.Tusas(mesh, prm, stream=stream)
    h.set_state(Ustart, t_start, dt)
    h.timers(True)
    secs, st = _steps_timed(h, n, stream)
    tm = h.get_timers()
    h.close()
    return {"s_per_step": secs, "mean_s_per_step": sum(secs) / n,
            "newton_its": [s["newton_its"] for s in st], "gmres_its": [s["gmres_its"] for s in st],
            "converged": all(s["converged"] for s in st),
            "timers_ms": {k: round(v[0], 3) for k, v in tm.items()}}


def run_ours(args, ws, rank, local):
    import dataclasses

    import torch

    import paper_2006_16764_b300 as pkg

    assert torch.cuda.is_available(), "bench needs a CUDA device"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.workload(args.workload)
    prm = w.params
    mesh = w.mesh
    N = mesh.n_dofs
    ne = mesh.n_elems
    nn = mesh.n_nodes
    U0 = torch.tensor(synth.initial_state(w), device=dev)
    stream = torch.cuda.current_stream(dev)
    fp64_peak, fp32_peak = pkg.fma_peak()
    hbm_peak, hbm_kind = _hbm_peak()
    h = pkg.Tusas(mesh, prm, stream=stream)
    h.set_state(U0, 0.0, w.dt)
    for _ in range(args.warmup):
        h.step()
    Ustart = torch.empty_like(U0)
    h.get_state(Ustart)
    t_start = h.time

    # ---- timed region: `steps` implicit time steps (the whole hot path) ----
    h.timers(True)
    l0 = pkg.kernel_launches()
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize(dev)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    stats = []
    for i in range(args.steps):
        stats.append(h.step())
        ev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    step_launches = pkg.kernel_launches() - l0
    step_s = [ev[i].elapsed_time(ev[i + 1]) / 1e3 for i in range(args.steps)]
    ms = ev[0].elapsed_time(ev[-1])
    ms_max = allreduce_max(ws, ms, dev)
    timers = h.get_timers()

    # ---- the headline: isolated residual evaluations of the converged state ----
    Ut = torch.empty_like(U0)
    h.get_state(Ut)
    F = torch.empty_like(U0)
    for _ in range(3):
        h.residual(Ut, F)
    l1 = pkg.kernel_launches()
    barrier(ws)
    torch.cuda.synchronize(dev)
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(args.steps):
        h.residual(Ut, F)
    r1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    clk = clocks.stop()
    res_launches = pkg.kernel_launches() - l1
    res_ms = r0.elapsed_time(r1)
    res_ms_max = allreduce_max(ws, res_ms, dev)
    value = allreduce_sum(ws, float(args.steps) * N, dev) / (res_ms_max * 1e-3) / 1e6
    res_per = res_ms / args.steps
    residual_kernel = {
        "ms": res_per, "Mdof_evals_per_s": N / (res_per * 1e-3) / 1e6,
        "kernel": "res3_kernel<1,0> (3D alloy residual), one evaluation = 8 colour launches",
        "fp64": {"achieved_tflops": FP64_FLOPS_PER_ELEM["residual"] * ne / (res_per * 1e-3) / 1e12,
                 "peak_tflops": fp64_peak / 1e12,
                 "frac": FP64_FLOPS_PER_ELEM["residual"] * ne / (res_per * 1e-3) / fp64_peak,
                 "issue_frac": FP64_PIPE_SLOTS_PER_ELEM["residual"] * ne / (res_per * 1e-3) / (fp64_peak / 2),
                 "basis": "FP64-pipe slots per element measured on this box and state (ncu, %.1f); flops "
                          "from them with the profiling box's flops per slot (estimate)" % FP64_PIPE_SLOTS_PER_ELEM["residual"]},
        "hbm": {"algorithmic_bytes": ALG_BYTES_PER_NODE["residual"] * nn,
                "achieved_gbs": ALG_BYTES_PER_NODE["residual"] * nn / (res_per * 1e-3) / 1e9,
                "peak_gbs": hbm_peak, "peak_kind": hbm_kind},
        "measured_dram_bytes": NCU_BYTES_PER_ELEM["residual"] * ne}
    residual_kernel["hbm"]["frac"] = residual_kernel["hbm"]["achieved_gbs"] / hbm_peak

    # ---- dominant kernel of the time step and its roofline ----
    dom = max(("residual", "residual_lin", "jv"), key=lambda k: timers[k][0])
    d_ms, d_cnt = timers[dom]
    per_launch = d_ms / max(d_cnt, 1)
    flops = FP64_FLOPS_PER_ELEM[dom] * ne
    achieved = flops / (per_launch * 1e-3) / 1e12
    alg_bytes = ALG_BYTES_PER_NODE[dom] * nn
    roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved * 1e12 / fp64_peak, "traffic": NCU_BYTES_PER_ELEM[dom] * ne,
            "kernel": ("tan3_kernel<1,false> (3D alloy tangent J v)" if dom == "jv" else f"res3_kernel {dom} (3D alloy)")
            + ", one operator application = 8 colour launches",
            "launch_ms": per_launch, "launches": d_cnt,
            "peak_kind": "FP64 FMA-chain throughput measured in this run (tusas_fma_peak)",
            "fp64_issue_frac": FP64_PIPE_SLOTS_PER_ELEM[dom] * ne / (per_launch * 1e-3) / (fp64_peak / 2),
            "hbm": {"algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / (per_launch * 1e-3) / 1e9,
                    "peak_gbs": hbm_peak, "peak_kind": hbm_kind,
                    "basis": "nodal vectors only (48 B/node for F, 64 B/node for J v)"},
            "design_lever": {"stored_linearisation_bytes": LIN_BYTES_PER_ELEM * ne,
                             "what": "the pointwise Jacobian read by every exact J v (written once per Newton "
                                     "iteration): HBM traffic traded for FP64 work, not algorithmic bytes",
                             "measured_dram_bytes": NCU_BYTES_PER_ELEM[dom] * ne}}
    roof["hbm"]["frac"] = roof["hbm"]["achieved_gbs"] / hbm_peak

    # ---- exact + FP32 against FD + FP64 over the same steps, at the workload's cap and at 30 ----
    jfnk = {"exact_fp32": {"s_per_step": ms / args.steps / 1e3, "steps_per_s": args.steps * 1e3 / ms,
                           "per_step_s": step_s,
                           "newton_its": [s["newton_its"] for s in stats],
                           "gmres_its": [s["gmres_its"] for s in stats],
                           "operator_evals_Mdof_per_s": sum(s["residual_evals"] + s["jv_evals"] for s in stats)
                           * N / (ms * 1e-3) / 1e6,
                           "kappa": 2 * w.dt * (prm.D / (1 + prm.k)) / mesh.h ** 2}}
    nfd = min(args.fd_steps, args.steps)
    if nfd > 0:
        pfd = dataclasses.replace(prm, jvp_mode=0, smoother_fp32=0)
        fd = _arm(pkg, mesh, pfd, Ustart, t_start, w.dt, nfd, stream)
        ex_win = step_s[:nfd]
        jfnk["fd_fp64"] = fd
        jfnk["same_window"] = {
            "steps": nfd, "from": "the state after the warm-up steps (both arms)",
            "exact_fp32_mean_s": sum(ex_win) / nfd, "fd_fp64_mean_s": fd["mean_s_per_step"],
            "speedup_exact_fp32_over_fd_fp64": fd["mean_s_per_step"] / (sum(ex_win) / nfd)}
    if args.cap30_steps > 0:
        c30 = {}
        for name, over in (("exact_fp32", dict(jvp_mode=1, smoother_fp32=1)),
                           ("fd_fp64", dict(jvp_mode=0, smoother_fp32=0))):
            c30[name] = _arm(pkg, mesh, dataclasses.replace(prm, gmres_maxit=30, **over), Ustart, t_start, w.dt,
                             args.cap30_steps, stream)
        c30["speedup_exact_fp32_over_fd_fp64"] = (c30["fd_fp64"]["mean_s_per_step"]
                                                  / c30["exact_fp32"]["mean_s_per_step"])
        c30["note"] = "gmres_maxit 30: one full GMRES(30) cycle per Newton iteration, same start state and steps"
        jfnk["gmres_cap_30"] = c30

    # ---- end to end through the C-ABI with pinned host buffers ----
    e2e = None
    if args.e2e_steps > 0:
        # the headline metric: per evaluation, H2D of its U from pinned host memory, the
        # residual, D2H of its F to pinned host memory. Double-buffered on three streams
        # (copy in, compute on the handle's stream, copy out): evaluation i computes while
        # the input of i + 1 and the output of i - 1 move, as a stream of evaluations would.
        Uh = [torch.empty(N, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        Fh = [torch.empty(N, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        for b in range(2):
            Uh[b].copy_(Ut.cpu())
        Ud = [torch.empty_like(U0) for _ in range(2)]
        Fd = [torch.empty_like(U0) for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ne2e = max(args.e2e_evals, 1)
        ev_in = [torch.cuda.Event() for _ in range(ne2e)]
        ev_c = [torch.cuda.Event() for _ in range(ne2e)]
        ev_out = [torch.cuda.Event() for _ in range(ne2e)]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(ne2e):
            b = i % 2
            if i >= 2:
                s_in.wait_event(ev_c[i - 2])  # Ud[b] is free once evaluation i - 2 is done
            with torch.cuda.stream(s_in):
                Ud[b].copy_(Uh[b], non_blocking=True)
            ev_in[i].record(s_in)
            stream.wait_event(ev_in[i])
            if i >= 2:
                stream.wait_event(ev_out[i - 2])  # Fd[b] is free once copied out
            h.residual(Ud[b], Fd[b])
            ev_c[i].record(stream)
            s_out.wait_event(ev_c[i])
            with torch.cuda.stream(s_out):
                Fh[b].copy_(Fd[b], non_blocking=True)
            ev_out[i].record(s_out)
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        ok = bool(torch.equal(Fh[(ne2e - 1) % 2], F.cpu()))  # same state, bitwise the same F
        e2e = {"value": ne2e * N / el / 1e6, "unit": UNIT, "h2d_bytes_per_step": 8 * N,
               "d2h_bytes_per_step": 8 * N, "steps": ne2e, "output_matches_device_run": ok,
               "what": "tusas_residual from pinned host U to pinned host F, host clock, copies of "
                       "neighbouring evaluations overlapped with compute (double-buffered, 3 streams); "
                       "the first copy in and the last copy out are not overlapped"}
        # the time step end to end: state in, step, state out
        Sh = torch.empty(N, dtype=torch.float64, pin_memory=True)
        Sh.copy_(Ustart.cpu())
        torch.cuda.synchronize(dev)
        tt = t_start
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            h.set_state(Sh, tt, w.dt)
            h.step()
            h.get_state(Sh)
            tt += w.dt
        el = time.perf_counter() - t0
        e2e["time_step"] = {"s_per_step": el / args.e2e_steps, "steps": args.e2e_steps,
                            "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N}

    line = None
    if rank == 0:
        cpu_rate, n1, el1, wsub = cpu_oracle_rate(args.cpu_seconds / 3, warm=1)
        pool = OraclePool()
        mc_rate, mc_n, mc_el, spread = pool.rate(2 * args.cpu_seconds / 3)
        pool.close()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(w, ws),
            "value_def": VALUE_DEF,
            "roofline": roof,
            "residual_kernel": residual_kernel,
            "cpu_baseline": {"value": mc_rate, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "sample": f"numpy oracle residual on the {CPU_SAMPLE[0]}x{CPU_SAMPLE[1]}x{CPU_SAMPLE[2]} "
                                       f"sub-box ({wsub.mesh.n_dofs} dofs), median of {mc_n} evaluations "
                                       f"({mc_el:.1f} s), element chunks over {pool.procs} spawned processes",
                             "spread_s": spread,
                             "single_core": {"value": cpu_rate, "cores": 1, "evaluations": n1, "seconds": el1}},
            "e2e": e2e,
            "gpu_launches": step_launches + res_launches,
            "gpu_launches_split": {"time_steps": step_launches, "residual_evals": res_launches},
            "clocks": clk,
            "jfnk": jfnk,
            "timers_ms": {k: [round(v[0], 3), v[1]] for k, v in timers.items()},
            "fp64_fma_peak_tflops": fp64_peak / 1e12, "fp32_fma_peak_tflops": fp32_peak / 1e12,
        }
        print(json.dumps(line), flush=True)
    h.close()


def main():
    args = parse()
    if args.kernels:
        run_kernels(args.kernels)
        return
    if args.report:
        run_report(args.report)
        return
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
