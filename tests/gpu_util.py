"""Helpers of the GPU tests: handles from synthetic workloads, host/device copies, norms."""
import numpy as np


def torch_cuda():
    import torch

    return torch


def dev(x):
    torch = torch_cuda()
    return torch.tensor(np.ascontiguousarray(x), device="cuda", dtype=torch.float64)


def host(t):
    torch = torch_cuda()
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    """Normwise relative error ||a - b||_inf / ||b||_inf."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def handle(mesh, prm):
    import paper_2006_16764_b300 as pkg

    return pkg.Tusas(mesh, prm)
