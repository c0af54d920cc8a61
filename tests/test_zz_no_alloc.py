"""The allocation-free reduction entry point against the handle-based one.

tusas_multidot_noalloc is for callers that cannot allocate device memory at
the point where they need a dot product (all memory given to their own pool,
no room for cudaMalloc's implicit synchronisation, or no handle allowed). It
must return what tusas_dot returns. Collected last (file name) so that a run
stopping at the first failure has already run every other test; it also
passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from synth import Mesh, Params

pytestmark = pytest.mark.gpu


def _call(lib, X, ld, k, y, n):
    out = (ctypes.c_double * max(k, 1))()
    rc = lib.tusas_multidot_noalloc(ctypes.c_void_p(X.data_ptr()), ld, k, ctypes.c_void_p(y.data_ptr()), n, out, None)
    return rc, [out[j] for j in range(k)]


def test_noalloc_dot_matches_tusas_dot_on_two_calls():
    import torch

    import paper_2006_16764_b300 as pkg

    lib = pkg.lib()
    mesh = Mesh(3, 23, 17, 11, 0.8)
    n = mesh.n_dofs
    k = 5
    X = torch.tensor(np.stack([synth.uniform_pm1(100 + j, n) for j in range(k)]), device="cuda").reshape(-1)
    y = torch.tensor(synth.uniform_pm1(7, n), device="cuda")
    h = pkg.Tusas(mesh, Params(model=0, precond=0))
    want = [h.dot(X[j * n:(j + 1) * n], y, n) for j in range(k)]
    torch.cuda.synchronize()
    free0 = None
    for call in range(2):  # the shared scratch keeps the previous call's contents
        rc, got = _call(lib, X, n, k, y, n)
        assert rc == pkg.OK
        # same partition and summation order as tusas_dot: bitwise equal, for every k
        assert got == want
        rc, got1 = _call(lib, X, n, 1, y, n)
        assert rc == pkg.OK and got1[0] == want[0]
        torch.cuda.synchronize()
        free = torch.cuda.mem_get_info()[0]
        if call == 0:
            free0 = free
        else:
            assert free == free0, "the second call changed the free device memory"
    # the Python wrapper is the same call
    assert pkg.multidot_noalloc(X, 2, y, n)[1] == got[1]
    h.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch

    import paper_2006_16764_b300 as pkg

    lib = pkg.lib()
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    X = torch.zeros(8 * 40, dtype=torch.float64, device="cuda")
    rc, _ = _call(lib, X, 8, pkg.NOALLOC_MAX_K + 1, y, 8)
    assert rc == pkg.EINVAL
    rc, _ = _call(lib, X, 8, 0, y, 8)
    assert rc == pkg.EINVAL
    rc, got = _call(lib, X, 8, pkg.NOALLOC_MAX_K, y, 8)
    assert rc == pkg.OK and got == [0.0] * pkg.NOALLOC_MAX_K
