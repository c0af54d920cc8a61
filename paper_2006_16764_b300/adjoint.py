"""Discrete-adjoint gradients of the final solid fraction behind a torch.autograd.Function.

S(eps4, Delta) = int (1 + phi_N)/2 after N backward-Euler steps. The forward
sweep (tusas_forward) records checkpoints; S and its weights dS/dU_N come from
tusas_solid_fraction; backward (tusas_adjoint) solves the transposed
linearised steps in reverse with the library's J^T w kernels and contracts
with dF/d eps4 and with dU_0/dDelta. Only argument marshalling here.
"""
from __future__ import annotations

import dataclasses

import torch


class SolidFraction(torch.autograd.Function):
    """S = SolidFraction.apply(eps4, Delta, problem); eps4 and Delta are 0-d float64 tensors.

    ``problem`` holds the handle, base parameters, the initial state as a
    function of Delta (device tensor), dU_0/dDelta (device tensor), t0, dt,
    nsteps, ckpt_every.
    """

    @staticmethod
    def forward(ctx, eps4, delta, problem):
        pb = problem
        prm = dataclasses.replace(pb.params, eps4=float(eps4), Delta=float(delta))
        pb.handle.set_params(prm)
        U0 = pb.initial_state(float(delta))
        pb.last_forward = pb.handle.forward(U0, pb.t0, pb.dt, pb.nsteps, pb.ckpt_every)
        UN = torch.empty_like(U0)
        pb.handle.get_state(UN)
        S = pb.handle.solid_fraction(UN)
        ctx.problem = pb
        return torch.tensor(S, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gS):
        pb = ctx.problem
        ge, gd, st = pb.handle.adjoint(pb.weights(), pb.dU0_ddelta, rtol=pb.adj_rtol)
        pb.last_adjoint = st
        g = gS.detach().to(torch.float64).cpu()
        return g * ge, g * gd, None


@dataclasses.dataclass
class SolidFractionProblem:
    handle: object
    params: object
    initial_state: object  # Delta -> device tensor U_0
    dU0_ddelta: torch.Tensor
    t0: float
    dt: float
    nsteps: int
    ckpt_every: int
    adj_rtol: float = 1e-10
    last_forward: dict = None
    last_adjoint: dict = None
    stream: object = None  # the handle's torch.cuda.Stream (solid_fraction_batch)
    w: torch.Tensor = None  # dS/dU_N from the library, filled on first use

    def weights(self):
        if self.w is None:
            self.w = self.handle.solid_fraction_weights(torch.empty_like(self.dU0_ddelta))
        return self.w


def solid_fraction_batch(problems, samples):
    """S and its discrete-adjoint gradients for several (eps4, Delta) samples at once.

    Problem i (its own handle, created on its own stream ``problems[i].stream``)
    takes ``samples[i]``; one host thread drives each handle, so the kernels of
    all samples share the GPU (the library releases the interpreter lock in
    every call and keeps no global state between handles). Returns a list of
    dicts with S, dS/d eps4, dS/d Delta and the forward / adjoint statistics;
    each sample gives bitwise the same numbers as a sequential run.
    """
    from concurrent.futures import ThreadPoolExecutor

    torch.cuda.synchronize()

    def one(pb, sample):
        e4, dl = float(sample[0]), float(sample[1])
        with torch.cuda.stream(pb.stream):
            prm = dataclasses.replace(pb.params, eps4=e4, Delta=dl)
            pb.handle.set_params(prm)
            U0 = pb.initial_state(dl)
            fw = pb.handle.forward(U0, pb.t0, pb.dt, pb.nsteps, pb.ckpt_every)
            UN = torch.empty_like(U0)
            pb.handle.get_state(UN)
            S = pb.handle.solid_fraction(UN)
            ge, gd, st = pb.handle.adjoint(pb.weights(), pb.dU0_ddelta, rtol=pb.adj_rtol)
        return {"eps4": e4, "Delta": dl, "S": S, "dS_deps4": ge, "dS_dDelta": gd, "forward": fw, "adjoint": st}

    with ThreadPoolExecutor(max_workers=len(problems)) as ex:
        return list(ex.map(one, problems, samples))
