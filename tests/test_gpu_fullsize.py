"""Converged steps at the full workload sizes, in the configuration the bench times.

The oracle cannot solve these sizes, so the GPU's first converged step is checked
by properties that hold at any size:

* the oracle's own residual, evaluated node by node at sampled nodes of the GPU
  state, is at the Newton tolerance (|F_i| <= ||F||_2 of the GPU's final iterate,
  plus roundoff relative to the initial residual at the same nodes);
* the conserved integral of the u equation (pure metal: int (u - phi/2); alloy:
  int A(phi) B(u) / (1 - k)) changes by at most dt sqrt(N) ||F||_2, because
  sum_i R_u,i is its exact difference quotient (consistent Q1 mass, applied here
  by 1D factors along each axis);
* a centred seed keeps the square symmetry of the 2D dendrite;
* the FP64 V-cycle is symmetric, and the FP32 one stays within the FP32 bound of it.
"""
import dataclasses
import math

import numpy as np
import pytest

import synth
from synth import Mesh, Params
from oracle import residual as OR
from tests.gpu_util import dev, handle, host

pytestmark = pytest.mark.gpu


def _mass_apply(mesh, v):
    """Consistent Q1 mass matrix times a nodal field, one tridiagonal 1D factor per axis."""
    shape = (mesh.nz + 1, mesh.ny + 1, mesh.nx + 1) if mesh.dim == 3 else (mesh.ny + 1, mesh.nx + 1)
    a = v.reshape(shape).copy()
    for ax in range(a.ndim):
        b = np.moveaxis(a, ax, 0)
        out = 4.0 * b
        out[1:] += b[:-1]
        out[:-1] += b[1:]
        out[0] -= 2.0 * b[0]
        out[-1] -= 2.0 * b[-1]
        a = np.moveaxis(out * (mesh.h / 6.0), 0, ax)
    return a.reshape(-1)


def _conserved(mesh, prm, V):
    n = mesh.n_nodes
    phi, u = V[:n], V[n:]
    if prm.model == 0:
        return float(np.sum(_mass_apply(mesh, u - phi / 2)))
    k = prm.k
    A = ((1 + k) - (1 - k) * phi) / 2
    return float(A @ _mass_apply(mesh, 1 + (1 - k) * u)) / (1 - k)


@pytest.mark.parametrize("name", ["dendrite2d_1024", "dendrite3d_192", "alloy3d_256x256x128"])
def test_full_size_first_step(name):
    w = synth.workload(name)
    mesh, prm = w.mesh, w.params
    U0 = synth.initial_state(w)
    h = handle(mesh, prm)
    h.set_state(dev(U0), 0.0, w.dt)
    st = h.step()
    assert st["converged"], st
    U1 = host(h.get_state(dev(np.zeros_like(U0))))
    n = mesh.n_nodes
    picks = (synth.splitmix64(11, 40) % np.uint64(n)).astype(np.int64)
    nodes = np.unique(np.concatenate([picks, [0, n - 1, n // 2]]))
    r0p, r0u = OR.residual_at_nodes(mesh, prm, U0, U0, 0.0, w.dt, nodes)
    r1p, r1u = OR.residual_at_nodes(mesh, prm, U1, U0, 0.0, w.dt, nodes)
    scale = max(np.abs(r0p).max(), np.abs(r0u).max())
    assert max(np.abs(r1p).max(), np.abs(r1u).max()) <= 1.01 * st["fnorm"] + 1e-12 * scale
    I0, I1 = _conserved(mesh, prm, U0), _conserved(mesh, prm, U1)
    assert abs(I1 - I0) <= 1.001 * w.dt * math.sqrt(n) * st["fnorm"] + 1e-12 * abs(I0)


def test_centred_seed_keeps_square_symmetry():
    """10 steps of a centred 2D seed (256^2, exact tangent, FP32 multigrid)."""
    L = 0.8 * 256
    mesh = Mesh(2, 256, 256, 0, 0.8, -L / 2, -L / 2)
    prm = Params(model=0, eps4=0.05, lam=3.19, D=2.0, Delta=0.65, precond=2, jvp_mode=1, smoother_fp32=1,
                 gmres_maxit=30)
    U = synth.seed_state(mesh, prm, radius=10.0, centred=True)
    h = handle(mesh, prm)
    h.set_state(dev(U), 0.0, 0.5)
    for _ in range(10):
        assert h.step()["converged"]
    V = host(h.get_state(dev(np.zeros_like(U))))
    n = mesh.n_nodes
    for f in (V[:n], V[n:]):
        g = f.reshape(257, 257)  # [j, i]
        scale = np.abs(g).max()
        assert np.abs(g - g.T).max() < 1e-8 * scale
        assert np.abs(g - g[:, ::-1]).max() < 1e-8 * scale
        assert np.abs(g - g[::-1, :]).max() < 1e-8 * scale


def test_full_size_vcycle_symmetric_and_fp32_close():
    """The block-Jacobi V-cycle on the full alloy box (its 33 x 33 x 17 coarsest level takes the
    3-blocks-per-SM smoother build). In FP64 it is symmetric to roundoff: the same Chebyshev
    polynomial in D^-1 A smooths before and after the coarse correction, restriction is P^T,
    and the coarsest level's sweeps are a polynomial in D^-1 A too. The FP32 cycle stays within
    the bound of the oracle comparison (2e-4 normwise) of the FP64 one."""
    w = synth.workload("alloy3d_256x256x128")
    U0 = synth.initial_state(w)
    U = U0 + 0.01 * synth.random_vector(w.mesh, 3)
    v = synth.random_vector(w.mesh, 21)
    z = synth.random_vector(w.mesh, 22)
    out = {}
    for fp32 in (0, 1):
        prm = dataclasses.replace(w.params, precond=2, smoother_fp32=fp32)
        h = handle(w.mesh, prm)
        h.set_state(dev(U0), 0.0, w.dt)
        h.precond_setup(dev(U))
        Mv, Mz = dev(np.zeros_like(v)), dev(np.zeros_like(z))
        h.precond_apply(dev(v), Mv)
        h.precond_apply(dev(z), Mz)
        out[fp32] = (host(Mv).copy(), host(Mz).copy())
        h.close()
    Mv, Mz = out[0]
    assert abs(v @ Mz - z @ Mv) <= 1e-12 * (np.abs(v) @ np.abs(Mz))
    for a, b in zip(out[1], out[0]):
        assert np.linalg.norm(a - b) <= 2e-4 * np.linalg.norm(b)
