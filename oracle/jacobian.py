"""Derivatives of the oracle residual by the complex-step method.

The Jacobian F'(U)_ij = dF_i/dU_j (Sec. 2.2) is never written out by hand
here: every derivative is the imaginary part of the residual evaluated at a
complex perturbation of size 1e-30 (Squire and Trapp 1998; Martins, Sturdza
and Alonso 2003), exact to roundoff because no subtraction occurs. This pins
the GPU's hand-written tangent and adjoint against the plain definition.

* ``jvp``               F'(U) v
* ``element_jacobians`` the element Jacobians (E, 2, 2^d, 2, 2^d)
* ``sparse_jacobian``   assembled F'(U) (scipy CSR)
* ``jtvp``              F'(U)^T w via the element Jacobians
* ``dF_deps4``          dF/d eps4
* ``dF_dUn_T``          (dF/dU^n)^T w, the coupling of consecutive time steps
* ``jvp_at_nodes``, ``jtvp_at_nodes``  the same products at listed nodes only,
  from the elements adjacent to them (for meshes too large to evaluate whole)

Parity: pinned against brute-force central differences (tests/test_oracle_jacobian.py).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import fem
from .residual import element_residual, gather, residual, residual_at_nodes

H_CS = 1e-30


def jvp(mesh, prm, U, Un, t_n, dt, v, Unm1=None):
    return residual(mesh, prm, U + 1j * H_CS * v, Un, t_n, dt, Unm1=Unm1).imag / H_CS


def dF_deps4(mesh, prm, U, Un, t_n, dt):
    p = dataclasses.replace(prm, eps4=prm.eps4 + 1j * H_CS)
    return residual(mesh, p, U.astype(complex), Un, t_n, dt).imag / H_CS


def element_jacobians(mesh, prm, U, Un, t_n, dt, elems=None, wrt_prev=False, Unm1=None):
    """dRe/dUe per element: (E, 2, 2^d, 2, 2^d) indexed [field_i, a, field_j, b].

    With ``wrt_prev`` the derivative is taken with respect to U^n instead of U.
    """
    if elems is None:
        elems = fem.all_elements(mesh)
    conn = fem.connectivity(mesh, elems)
    phi_e, u_e = gather(mesh, U, conn)
    phin_e, un_e = gather(mesh, Un, conn)
    pm1_e = gather(mesh, Unm1, conn)[0] if Unm1 is not None else None
    E, nl = conn.shape
    Je = np.zeros((E, 2, nl, 2, nl))
    for fj in range(2):
        for b in range(nl):
            pert = np.zeros((E, nl), dtype=complex)
            pert[:, b] = 1j * H_CS
            args = [phi_e.astype(complex), u_e.astype(complex), phin_e.astype(complex), un_e.astype(complex)]
            idx = fj + (2 if wrt_prev else 0)
            args[idx] = args[idx] + pert
            c = element_residual(mesh, prm, elems, *args, t_n, dt, None, pm1_e)
            Je[:, :, :, fj, b] = c.imag / H_CS
    return Je, conn


def sparse_jacobian(mesh, prm, U, Un, t_n, dt, wrt_prev=False, Unm1=None):
    n = mesh.n_nodes
    Je, conn = element_jacobians(mesh, prm, U, Un, t_n, dt, wrt_prev=wrt_prev, Unm1=Unm1)
    E, nl = conn.shape
    rows = np.empty((E, 2, nl, 2, nl), dtype=np.int64)
    cols = np.empty_like(rows)
    for fi in range(2):
        for a in range(nl):
            for fj in range(2):
                for b in range(nl):
                    rows[:, fi, a, fj, b] = fi * n + conn[:, a]
                    cols[:, fi, a, fj, b] = fj * n + conn[:, b]
    J = sp.coo_matrix((Je.reshape(-1), (rows.reshape(-1), cols.reshape(-1))), shape=(2 * n, 2 * n))
    return J.tocsr()


def jtvp(mesh, prm, U, Un, t_n, dt, w, wrt_prev=False, Unm1=None):
    """(dF/dU)^T w, or (dF/dU^n)^T w with ``wrt_prev``, summed element by element."""
    n = mesh.n_nodes
    Je, conn = element_jacobians(mesh, prm, U, Un, t_n, dt, wrt_prev=wrt_prev, Unm1=Unm1)
    we = np.stack([w[:n][conn], w[n:][conn]], axis=1)  # (E, 2, nl)
    contrib = np.einsum("eiajb,eia->ejb", Je, we)
    out = np.zeros(2 * n)
    out[:n] = fem.scatter_add(n, conn, contrib[:, 0, :])
    out[n:] = fem.scatter_add(n, conn, contrib[:, 1, :])
    return out


def dF_dUn_T(mesh, prm, U, Un, t_n, dt, w):
    return jtvp(mesh, prm, U, Un, t_n, dt, w, wrt_prev=True)


def jvp_at_nodes(mesh, prm, U, Un, t_n, dt, v, nodes):
    """(F'(U) v) at the listed nodes: the complex step of residual_at_nodes, (rows phi, rows u)."""
    rp, ru = residual_at_nodes(mesh, prm, U + 1j * H_CS * v, Un, t_n, dt, nodes)
    return rp.imag / H_CS, ru.imag / H_CS


def jtvp_at_nodes(mesh, prm, U, Un, t_n, dt, w, nodes):
    """(F'(U)^T w) at the listed nodes: column j of F' meets w only on the elements adjacent to
    node j, so their element Jacobians give the entries exactly; (entries phi, entries u)."""
    n = mesh.n_nodes
    nodes = np.asarray(nodes, dtype=np.int64)
    elems = fem.elements_of_nodes(mesh, nodes)
    Je, conn = element_jacobians(mesh, prm, U, Un, t_n, dt, elems=elems)
    we = np.stack([w[:n][conn], w[n:][conn]], axis=1)  # (E, 2, nl)
    contrib = np.einsum("eiajb,eia->ejb", Je, we)
    pos = {int(v): i for i, v in enumerate(nodes)}
    out_p = np.zeros(len(nodes))
    out_u = np.zeros(len(nodes))
    for e in range(conn.shape[0]):
        for b in range(conn.shape[1]):
            i = pos.get(int(conn[e, b]))
            if i is not None:
                out_p[i] += contrib[e, 0, b]
                out_u[i] += contrib[e, 1, b]
    return out_p, out_u
