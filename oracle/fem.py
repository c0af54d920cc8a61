"""Q1 finite elements on a structured box (Sec. 2.1.1: Lagrange nodal Q1 quads / hexes).

Element e = (ei, ej[, ek]) has local node a = ax + 2 ay (+ 4 az) at global node
(ei+ax, ej+ay[, ek+az]); global node index i + (nx+1)(j + (ny+1) k).
Quadrature: tensor 2-point Gauss rule per axis (exact for the cubic-in-each-axis
products that Q1 mass and stiffness integrals produce).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def n_nodes_axis(mesh):
    return [mesh.nx + 1, mesh.ny + 1] + ([mesh.nz + 1] if mesh.dim == 3 else [])


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


def local_offsets(dim):
    """Offsets (ax, ay[, az]) of the 2^dim local nodes, local index a = ax + 2ay + 4az."""
    return [tuple((a >> d) & 1 for d in range(dim)) for a in range(2 ** dim)]


def connectivity(mesh, elems):
    """Global node numbers (E, 2^dim) of the given elements (dim, E)."""
    offs = local_offsets(mesh.dim)
    cols = [node_index(mesh, [elems[d] + o[d] for d in range(mesh.dim)]) for o in offs]
    return np.stack(cols, axis=1)


def gauss_rule(dim):
    """2-point Gauss points in the unit cell [0,1]^dim and weights (sum 1).

    Returns a list of (xi tuple, weight) with the point index g = gx + 2gy + 4gz.
    """
    s = 1.0 / math.sqrt(3.0)
    pts1 = [(1.0 - s) / 2.0, (1.0 + s) / 2.0]
    return [(tuple(pts1[(g >> d) & 1] for d in range(dim)), 0.5 ** dim) for g in range(2 ** dim)]


def basis(dim, xi, h):
    """Q1 basis values N_a(xi) (2^dim,) and physical gradients (dim, 2^dim) at xi."""
    offs = local_offsets(dim)
    N = np.empty(2 ** dim)
    G = np.empty((dim, 2 ** dim))
    for a, o in enumerate(offs):
        f = [xi[d] if o[d] else 1.0 - xi[d] for d in range(dim)]
        df = [1.0 if o[d] else -1.0 for d in range(dim)]
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
    coords = node_coords(mesh, nodes)
    cand = []
    for off in itertools.product([-1, 0], repeat=mesh.dim):
        e = [coords[d] + off[d] for d in range(mesh.dim)]
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
