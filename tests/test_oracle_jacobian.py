"""Pins of the oracle's complex-step derivatives against brute-force central differences."""
import dataclasses

import numpy as np
import pytest

import synth
from synth import Mesh, Params
from oracle import jacobian as J
from oracle import residual as R

CASES = [
    (Mesh(2, 5, 4, 0, 0.7, 0.1, 0.2), Params(model=0, eps4=0.05, lam=3.19, D=2.0)),
    (Mesh(2, 4, 5, 0, 0.8), Params(model=1, k=0.15, eps4=0.02, lam=3.19, D=2.0, lT=30.0, Vp=0.2)),
    (Mesh(3, 3, 3, 4, 0.8), Params(model=1, k=0.15, eps4=0.02, lam=3.19, D=2.0, lT=30.0, Vp=0.2, jat_normalised=0)),
    (Mesh(3, 4, 3, 3, 0.9), Params(model=0, eps4=0.05, lam=3.19, D=2.0, time_form=1)),
]
IDS = ["2d-pure", "2d-alloy", "3d-alloy-jat0", "3d-pure-literal"]


def _fd(f, x, v, h=1e-6):
    return (f(x + h * v) - f(x - h * v)) / (2 * h)


@pytest.mark.parametrize("mesh,prm", CASES, ids=IDS)
def test_jvp_matches_central_differences(mesh, prm):
    U, Un = synth.random_fields(mesh, 3)
    v = synth.random_vector(mesh, 4)
    dt, tn = 0.3, 0.7
    jv = J.jvp(mesh, prm, U, Un, tn, dt, v)
    fd = _fd(lambda X: R.residual(mesh, prm, X, Un, tn, dt), U, v)
    assert np.abs(jv - fd).max() <= 1e-7 * np.abs(jv).max()


@pytest.mark.parametrize("mesh,prm", CASES, ids=IDS)
def test_sparse_jacobian_transpose_and_prev_state(mesh, prm):
    U, Un = synth.random_fields(mesh, 5)
    v = synth.random_vector(mesh, 6)
    w = synth.random_vector(mesh, 7)
    dt, tn = 0.3, 0.0
    Js = J.sparse_jacobian(mesh, prm, U, Un, tn, dt)
    jv = J.jvp(mesh, prm, U, Un, tn, dt, v)
    assert np.abs(Js @ v - jv).max() <= 1e-13 * np.abs(jv).max()
    jtw = J.jtvp(mesh, prm, U, Un, tn, dt, w)
    assert np.abs(Js.T @ w - jtw).max() <= 1e-13 * np.abs(jtw).max()
    # adjoint identity w.(J v) = (J^T w).v
    assert abs(w @ jv - jtw @ v) <= 1e-12 * abs(w) @ abs(jv)
    # derivative with respect to the previous state
    fd = _fd(lambda X: R.residual(mesh, prm, U, X, tn, dt), Un, v)
    jpv = J.sparse_jacobian(mesh, prm, U, Un, tn, dt, wrt_prev=True) @ v
    assert np.abs(jpv - fd).max() <= 1e-7 * np.abs(fd).max()
    assert abs(w @ jpv - J.dF_dUn_T(mesh, prm, U, Un, tn, dt, w) @ v) <= 1e-12 * (abs(w) @ abs(jpv))


@pytest.mark.parametrize("mesh,prm", CASES, ids=IDS)
def test_dF_deps4_matches_central_differences(mesh, prm):
    U, Un = synth.random_fields(mesh, 8)
    d = J.dF_deps4(mesh, prm, U, Un, 0.0, 0.4)
    h = 1e-6
    Fp = R.residual(mesh, dataclasses.replace(prm, eps4=prm.eps4 + h), U, Un, 0.0, 0.4)
    Fm = R.residual(mesh, dataclasses.replace(prm, eps4=prm.eps4 - h), U, Un, 0.0, 0.4)
    fd = (Fp - Fm) / (2 * h)
    assert np.abs(d - fd).max() <= 1e-7 * np.abs(d).max()


def test_dense_jacobian_columns_brute_force():
    """Every column of the assembled Jacobian against a central difference on a 4x4 mesh."""
    mesh = Mesh(2, 4, 4, 0, 0.9)
    prm = Params(model=1, k=0.15, eps4=0.03, lam=3.0, D=2.0)
    U, Un = synth.random_fields(mesh, 21)
    Jd = J.sparse_jacobian(mesh, prm, U, Un, 0.0, 0.5).toarray()
    for j in range(mesh.n_dofs):
        e = np.zeros(mesh.n_dofs)
        e[j] = 1.0
        col = _fd(lambda X: R.residual(mesh, prm, X, Un, 0.0, 0.5), U, e, 1e-5)
        assert np.abs(Jd[:, j] - col).max() <= 1e-7 * max(1.0, np.abs(col).max())


@pytest.mark.parametrize("mesh,prm", CASES, ids=IDS)
def test_products_at_listed_nodes_match_the_whole_mesh(mesh, prm):
    """J v and J^T w at a few nodes (corners, faces, interior) from their adjacent
    elements only: the entries of the whole-mesh products, which the tests above pin."""
    U, Un = synth.random_fields(mesh, 11)
    v = synth.random_vector(mesh, 12)
    w = synth.random_vector(mesh, 13)
    dt, tn = 0.3, 0.2
    n = mesh.n_nodes
    nodes = np.array([0, n - 1, 1, mesh.shape_nodes[0], n // 2, n // 3, n - 2])
    jv = J.jvp(mesh, prm, U, Un, tn, dt, v)
    jp, ju = J.jvp_at_nodes(mesh, prm, U, Un, tn, dt, v, nodes)
    assert np.abs(jp - jv[nodes]).max() <= 1e-13 * np.abs(jv).max()
    assert np.abs(ju - jv[n + nodes]).max() <= 1e-13 * np.abs(jv).max()
    jtw = J.jtvp(mesh, prm, U, Un, tn, dt, w)
    tp, tu = J.jtvp_at_nodes(mesh, prm, U, Un, tn, dt, w, nodes)
    assert np.abs(tp - jtw[nodes]).max() <= 1e-13 * np.abs(jtw).max()
    assert np.abs(tu - jtw[n + nodes]).max() <= 1e-13 * np.abs(jtw).max()
