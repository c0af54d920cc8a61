"""Lagrange finite elements on a structured box (Sec. 2.1.1: nodal Q1 quads / hexes and
biquadratic Q2 quads).

Order p (1 or 2): element e = (ei, ej[, ek]) has local node a = sum_d a_d (p+1)^d
at global node (p ei + ax, p ej + ay[, p ek + az]); global node index
i + nnx (j + nny k) with nn = p n + 1 nodes per axis.
Quadrature: tensor Gauss rule with p + 1 points per axis (2 points for Q1,
exact for the Q1 mass and stiffness products; 3 points for Q2, the 9-point
rule of Sec. 4.1).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def order(mesh):
    return getattr(mesh, "order", 1)


def n_nodes_axis(mesh):
    p = order(mesh)
    return [p * mesh.nx + 1, p * mesh.ny + 1] + ([p * mesh.nz + 1] if mesh.dim == 3 else [])


def n_elems_axis(mesh):
    return [mesh.nx, mesh.ny] + ([mesh.nz] if mesh.dim == 3 else [])


def node_index(mesh, idx):
    """Flat node index from per-axis integer arrays (x fastest)."""
    nn = n_nodes_axis(mesh)
    flat = np.asarray(idx[0]).astype(np.int64)
    stride = 1
    for d in range(1, mesh.dim):
        stride *= nn[d - 1]
        flat = flat + stride * np.asarray(idx[d]).astype(np.int64)
    return flat


def all_elements(mesh):
    """Per-axis element indices of every element, x fastest, shape (dim, E)."""
    ne = n_elems_axis(mesh)
    grids = np.meshgrid(*[np.arange(n) for n in ne], indexing="ij")
    return np.stack([g.transpose().reshape(-1) for g in grids])


def local_offsets(dim, p=1):
    """Offsets (ax, ay[, az]) of the (p+1)^dim local nodes, local index a = sum_d a_d (p+1)^d."""
    out = []
    for a in range((p + 1) ** dim):
        o, r = [], a
        for _ in range(dim):
            o.append(r % (p + 1))
            r //= p + 1
        out.append(tuple(o))
    return out


def connectivity(mesh, elems):
    """Global node numbers (E, (p+1)^dim) of the given elements (dim, E)."""
    p = order(mesh)
    offs = local_offsets(mesh.dim, p)
    cols = [node_index(mesh, [p * elems[d] + o[d] for d in range(mesh.dim)]) for o in offs]
    return np.stack(cols, axis=1)


def gauss_1d(p=1):
    """(points in [0,1], weights summing to 1) of the (p+1)-point Gauss rule."""
    if p == 1:
        s = 1.0 / math.sqrt(3.0)
        return [(1.0 - s) / 2.0, (1.0 + s) / 2.0], [0.5, 0.5]
    s = math.sqrt(3.0 / 5.0)
    return [(1.0 - s) / 2.0, 0.5, (1.0 + s) / 2.0], [5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0]


def gauss_rule(dim, p=1):
    """Tensor Gauss points in the unit cell [0,1]^dim and weights (sum 1).

    Returns a list of (xi tuple, weight) with the point index g = sum_d g_d (p+1)^d.
    """
    pts, wts = gauss_1d(p)
    rule = []
    for g in range((p + 1) ** dim):
        idx, r = [], g
        for _ in range(dim):
            idx.append(r % (p + 1))
            r //= p + 1
        rule.append((tuple(pts[i] for i in idx), float(np.prod([wts[i] for i in idx]))))
    return rule


def lagrange_1d(p, x):
    """Values and derivatives of the 1D Lagrange basis on the p + 1 equispaced nodes of [0,1]."""
    if p == 1:
        return [1.0 - x, x], [-1.0, 1.0]
    return ([2.0 * (x - 0.5) * (x - 1.0), -4.0 * x * (x - 1.0), 2.0 * x * (x - 0.5)],
            [4.0 * x - 3.0, 4.0 - 8.0 * x, 4.0 * x - 1.0])


def basis(dim, xi, h, p=1):
    """Basis values N_a(xi) ((p+1)^dim,) and physical gradients (dim, (p+1)^dim) at xi."""
    offs = local_offsets(dim, p)
    vals = [lagrange_1d(p, xi[d]) for d in range(dim)]
    nl = (p + 1) ** dim
    N = np.empty(nl)
    G = np.empty((dim, nl))
    for a, o in enumerate(offs):
        f = [vals[d][0][o[d]] for d in range(dim)]
        df = [vals[d][1][o[d]] for d in range(dim)]
        N[a] = np.prod(f)
        for d in range(dim):
            prod = df[d]
            for e in range(dim):
                if e != d:
                    prod *= f[e]
            G[d, a] = prod / h
    return N, G


def scatter_add(n, conn, vals):
    """out[conn[e, a]] += vals[e, a]; real and imaginary parts summed separately."""
    idx = conn.reshape(-1)
    v = vals.reshape(-1)
    if np.iscomplexobj(v):
        re = np.bincount(idx, weights=v.real, minlength=n)
        im = np.bincount(idx, weights=v.imag, minlength=n)
        return re + 1j * im
    return np.bincount(idx, weights=v, minlength=n)


def node_coords(mesh, nodes):
    """Per-axis integer coordinates of flat node indices."""
    nn = n_nodes_axis(mesh)
    rem = np.asarray(nodes, dtype=np.int64)
    out = []
    for d in range(mesh.dim):
        out.append(rem % nn[d])
        rem = rem // nn[d]
    return out


def elements_of_nodes(mesh, nodes):
    """Per-axis indices (dim, M) of every element adjacent to any of the nodes (unique)."""
    ne = n_elems_axis(mesh)
    p = order(mesh)
    coords = node_coords(mesh, nodes)
    cand = []
    for off in itertools.product([-1, 0], repeat=mesh.dim):
        # node i lies in elements floor(i/p) - 1 and floor(i/p) when i is a multiple of p, else floor(i/p)
        e = [coords[d] // p + off[d] for d in range(mesh.dim)]
        for d in range(mesh.dim):
            e[d] = np.where((coords[d] % p != 0) & (off[d] == -1), -1, e[d])
        ok = np.ones(len(coords[0]), dtype=bool)
        for d in range(mesh.dim):
            ok &= (e[d] >= 0) & (e[d] < ne[d])
        cand.append(np.stack([x[ok] for x in e]))
    allc = np.concatenate(cand, axis=1)
    flat = np.zeros(allc.shape[1], dtype=np.int64)
    stride = 1
    for d in range(mesh.dim):
        flat += stride * allc[d]
        stride *= ne[d]
    _, keep = np.unique(flat, return_index=True)
    return allc[:, np.sort(keep)]
