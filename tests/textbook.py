"""Textbook Q1 matrices on a structured box, built from 1D pieces (independent of the oracle).

1D linear elements of length h: element mass (h/6)[[2,1],[1,2]], element
stiffness (1/h)[[1,-1],[-1,1]]. The tensor-product Q1 space gives
M = M1 (x) M1 (x) M1 and K = sum over axes of K1 on that axis (x) M1 on the
others (Kronecker order with x fastest, i.e. the last factor is x).
"""
import numpy as np
import scipy.sparse as sp


def mass1(n, h):
    main = np.full(n + 1, 4.0)
    main[0] = main[-1] = 2.0
    off = np.ones(n)
    return sp.diags([off, main, off], [-1, 0, 1]) * (h / 6.0)


def stiff1(n, h):
    main = np.full(n + 1, 2.0)
    main[0] = main[-1] = 1.0
    off = -np.ones(n)
    return sp.diags([off, main, off], [-1, 0, 1]) * (1.0 / h)


def _kron_list(mats):
    out = mats[0]
    for m in mats[1:]:
        out = sp.kron(out, m)
    return out.tocsr()


def mass(mesh):
    ns = [mesh.nx, mesh.ny] + ([mesh.nz] if mesh.dim == 3 else [])
    m1 = [mass1(n, mesh.h) for n in ns]
    return _kron_list(m1[::-1])  # slowest axis first


def stiffness(mesh):
    ns = [mesh.nx, mesh.ny] + ([mesh.nz] if mesh.dim == 3 else [])
    total = None
    for d in range(mesh.dim):
        parts = [stiff1(n, mesh.h) if e == d else mass1(n, mesh.h) for e, n in enumerate(ns)]
        term = _kron_list(parts[::-1])
        total = term if total is None else total + term
    return total.tocsr()


def node_coords(mesh):
    """Coordinates (dim arrays) of all nodes in flat order (x fastest)."""
    c = mesh.coords()
    grids = np.meshgrid(*c, indexing="ij")
    return [np.ascontiguousarray(g.transpose()).reshape(-1) for g in grids]


def node_ijk(mesh):
    nn = list(mesh.shape_nodes)
    grids = np.meshgrid(*[np.arange(n) for n in nn], indexing="ij")
    return [np.ascontiguousarray(g.transpose()).reshape(-1) for g in grids]


def _assemble_1d(n, Ke):
    p = Ke.shape[0] - 1
    N = p * n + 1
    A = np.zeros((N, N))
    for e in range(n):
        A[p * e:p * e + p + 1, p * e:p * e + p + 1] += Ke
    return sp.csr_matrix(A)


def mass1_q2(n, h):
    """1D quadratic Lagrange mass matrix, element (h/30)[[4,2,-1],[2,16,2],[-1,2,4]]."""
    return _assemble_1d(n, (h / 30.0) * np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]))


def stiff1_q2(n, h):
    """1D quadratic Lagrange stiffness matrix, element (1/(3h))[[7,-8,1],[-8,16,-8],[1,-8,7]]."""
    return _assemble_1d(n, (1.0 / (3.0 * h)) * np.array([[7.0, -8.0, 1.0], [-8.0, 16.0, -8.0], [1.0, -8.0, 7.0]]))


def mass_q2(mesh):
    """Q2 (bi- or triquadratic) mass matrix: the Kronecker product of the 1D quadratic ones."""
    ns = [mesh.nx, mesh.ny] + ([mesh.nz] if mesh.dim == 3 else [])
    return _kron_list([mass1_q2(n, mesh.h) for n in ns][::-1])


def stiffness_q2(mesh):
    """Q2 stiffness matrix: per axis the 1D quadratic stiffness times the 1D masses of the others."""
    ns = [mesh.nx, mesh.ny] + ([mesh.nz] if mesh.dim == 3 else [])
    total = None
    for d in range(mesh.dim):
        parts = [stiff1_q2(n, mesh.h) if e == d else mass1_q2(n, mesh.h) for e, n in enumerate(ns)]
        term = _kron_list(parts[::-1])
        total = term if total is None else total + term
    return total.tocsr()
