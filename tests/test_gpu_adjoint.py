"""Discrete adjoint through N implicit steps on the GPU against the oracle adjoint
(direct solves) and central differences; checkpoint invariance; autograd wrapper."""
import dataclasses

import numpy as np
import pytest

import synth
from synth import Mesh, Params
from oracle import adjoint as OA
from tests.gpu_util import dev, handle, host

pytestmark = pytest.mark.gpu


def _problem(kind):
    if kind == "pure16":
        # the 16 x 16 case of the adjoint check against the oracle's direct-solve (dense Jacobian) adjoint
        mesh = Mesh(2, 16, 16, 0, 1.25)
        prm = Params(model=0, eps4=0.05, lam=3.19, D=2.0, Delta=0.65, precond=1, jvp_mode=1, newton_rtol=1e-13)
        U0f = lambda p: synth.seed_state(mesh, p, radius=8.0)
        return mesh, prm, U0f, 0.5, 3
    if kind == "alloy_cn":
        mesh = Mesh(2, 10, 10, 0, 1.2, -6.0, -6.0)
        prm = Params(model=1, k=0.15, eps4=0.03, lam=3.19, D=2.0, Delta=0.5, precond=1, jvp_mode=1,
                     newton_rtol=1e-13, theta=0.5, phihat_form=1)
        U0f = lambda p: synth.seed_state(mesh, p, radius=3.0, centred=True)
        return mesh, prm, U0f, 0.3, 3
    if kind == "pure":
        mesh = Mesh(2, 10, 10, 0, 2.0)
        prm = Params(model=0, eps4=0.04, lam=3.19, D=2.0, Delta=0.6, precond=1, jvp_mode=1, newton_rtol=1e-13)
        U0f = lambda p: synth.seed_state(mesh, p, radius=6.0)
        return mesh, prm, U0f, 0.5, 3
    mesh = Mesh(2, 10, 10, 0, 1.2, -6.0, -6.0)
    prm = Params(model=1, k=0.15, eps4=0.03, lam=3.19, D=2.0, Delta=0.5, precond=1, jvp_mode=1, newton_rtol=1e-13)
    U0f = lambda p: synth.seed_state(mesh, p, radius=3.0, centred=True)
    return mesh, prm, U0f, 0.3, 2


@pytest.mark.parametrize("kind", ["pure", "pure16", "alloy", "alloy_cn"])
def test_adjoint_matches_oracle_adjoint(kind):
    mesh, prm, U0f, dt, n = _problem(kind)
    U0 = U0f(prm)
    states = OA.forward(mesh, prm, U0, 0.0, dt, n)
    w, c = OA.solid_fraction_weights(mesh)
    g_eps, g0 = OA.gradient(mesh, prm, states, 0.0, dt, w)
    nn = mesh.n_nodes
    d0 = np.concatenate([np.zeros(nn), -np.ones(nn)])
    h = handle(mesh, prm)
    st = h.forward(dev(U0), 0.0, dt, n, 2)
    assert st["converged"]
    UN = host(h.get_state(dev(np.zeros_like(U0))))
    assert np.abs(UN - states[-1]).max() <= 1e-11 * np.abs(states[-1]).max()
    tg0 = dev(np.zeros_like(U0))
    ge, gd, ast = h.adjoint(dev(w), dev(d0), tg0, rtol=1e-12)
    # measured: dS/d eps4 within 3e-13 / 4e-13, dS/dU_0 within 9e-10 / 3e-13 (pure / alloy)
    assert abs(ge - g_eps) <= 1e-10 * abs(g_eps)
    assert abs(gd - g0 @ d0) <= 1e-8 * abs(g0 @ d0)
    assert np.abs(host(tg0) - g0).max() <= 1e-8 * np.abs(g0).max()
    # the state is restored to U_N
    assert np.array_equal(host(h.get_state(dev(np.zeros_like(U0)))), UN)


def test_checkpoint_spacing_does_not_change_the_gradient():
    mesh, prm, U0f, dt, _ = _problem("pure")
    U0 = dev(U0f(prm))
    w, _ = OA.solid_fraction_weights(mesh)
    h = handle(mesh, prm)
    res = []
    for every in (1, 2, 3, 5):
        h.forward(U0, 0.0, dt, 5, every)
        ge, gd, _ = h.adjoint(dev(w), None, None, rtol=1e-12)
        res.append(ge)
    assert max(res) - min(res) == 0.0, res


def test_autograd_function_matches_central_differences():
    import torch

    from paper_2006_16764_b300.adjoint import SolidFraction, SolidFractionProblem

    mesh, prm, U0f, dt, n = _problem("alloy")
    h = handle(mesh, prm)
    nn = mesh.n_nodes
    pb = SolidFractionProblem(h, prm, lambda d: dev(U0f(dataclasses.replace(prm, Delta=d))),
                              dev(np.concatenate([np.zeros(nn), -np.ones(nn)])), 0.0, dt, n, 1, 1e-12)
    eps = torch.tensor(prm.eps4, dtype=torch.float64, requires_grad=True)
    dl = torch.tensor(prm.Delta, dtype=torch.float64, requires_grad=True)
    S = SolidFraction.apply(eps, dl, pb)
    ge, gd = torch.autograd.grad(S, (eps, dl))
    hh = 1e-5

    def S_at(e, d):
        return float(SolidFraction.apply(torch.tensor(e, dtype=torch.float64), torch.tensor(d, dtype=torch.float64), pb))

    fd_e = (S_at(prm.eps4 + hh, prm.Delta) - S_at(prm.eps4 - hh, prm.Delta)) / (2 * hh)
    fd_d = (S_at(prm.eps4, prm.Delta + hh) - S_at(prm.eps4, prm.Delta - hh)) / (2 * hh)
    assert abs(float(ge) - fd_e) <= 1e-5 * abs(fd_e)
    assert abs(float(gd) - fd_d) <= 1e-5 * abs(fd_d)


def test_concurrent_samples_match_sequential_bitwise():
    """solid_fraction_batch: several samples on their own handles and streams at once give
    bitwise the numbers of one-at-a-time runs (deterministic kernels, no shared state)."""
    import torch

    import paper_2006_16764_b300 as pkg
    from paper_2006_16764_b300.adjoint import SolidFractionProblem, solid_fraction_batch

    mesh, prm, U0f, dt, n = _problem("alloy")
    w, _ = OA.solid_fraction_weights(mesh)
    nn = mesh.n_nodes
    d0 = dev(np.concatenate([np.zeros(nn), -np.ones(nn)]))
    init = lambda d: dev(U0f(dataclasses.replace(prm, Delta=d)))
    samples = [(0.03, 0.5), (0.045, 0.42), (0.02, 0.61)]
    probs = []
    for _ in samples:
        s = torch.cuda.Stream()
        probs.append(SolidFractionProblem(pkg.Tusas(mesh, prm, stream=s), prm, init, d0, 0.0, dt, n, 1, 1e-12,
                                          stream=s))
    seq = [solid_fraction_batch([pb], [sm])[0] for pb, sm in zip(probs, samples)]
    conc = solid_fraction_batch(probs, samples)
    for a, b in zip(seq, conc):
        assert (a["S"], a["dS_deps4"], a["dS_dDelta"]) == (b["S"], b["dS_deps4"], b["dS_dDelta"])
    # and the gradients are the oracle's
    st = OA.forward(mesh, dataclasses.replace(prm, eps4=0.045, Delta=0.42), U0f(dataclasses.replace(prm, Delta=0.42)),
                    0.0, dt, n)
    g_eps, g0 = OA.gradient(mesh, dataclasses.replace(prm, eps4=0.045, Delta=0.42), st, 0.0, dt, w)
    assert abs(conc[1]["dS_deps4"] - g_eps) <= 1e-10 * abs(g_eps)


@pytest.mark.parametrize("dim,order", [(2, 1), (3, 1), (2, 2), (3, 2)])
def test_solid_fraction_matches_oracle(dim, order):
    """tusas_solid_fraction: S and its weights against the oracle's exact integral of phi_h."""
    if dim == 2:
        mesh = Mesh(2, 7, 5, 0, 0.9, order=order)
    else:
        mesh = Mesh(3, 5, 4, 6, 0.8, order=order)
    prm = Params(model=0, precond=0)
    w, c = OA.solid_fraction_weights(mesh)
    U = synth.uniform_pm1(11, mesh.n_dofs)
    h = handle(mesh, prm)
    tw = h.solid_fraction_weights(dev(np.zeros(mesh.n_dofs)))
    assert np.abs(host(tw) - w).max() <= 1e-15 * np.abs(w).max()
    S = h.solid_fraction(dev(U))
    assert abs(S - (w @ U + c)) <= 1e-13 * abs(w @ U + c)
