"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/tusas.h.

No compute calls: this runs on machines without a GPU.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tusas.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tusas_[A-Za-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2006_16764_b300 import build

    build.build()
    import paper_2006_16764_b300 as pkg

    lib = pkg.lib()
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(pkg.EXPORTS) == names


def test_struct_layouts_match_header():
    """Field order of the ctypes mirrors equals the header's struct declarations."""
    import paper_2006_16764_b300 as pkg

    text = open(os.path.join(ROOT, "include", "tusas.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for cname, cls in (("tusas_params", pkg.CParams), ("tusas_mesh", pkg.CMesh), ("tusas_stats", pkg.CStats)):
        body = re.search(r"typedef struct %s \{(.*?)\}" % cname, text, re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            decl = re.sub(r"^(int|double)\s+", "", decl)
            for f in decl.split(","):
                fields.append(re.sub(r"\[.*\]", "", f).strip())
        assert [f for f, _ in cls._fields_] == fields, cname


def test_invalid_arguments_fail_without_gpu_work():
    """Argument validation happens before any CUDA call: null pointers are rejected."""
    import ctypes

    import paper_2006_16764_b300 as pkg

    lib = pkg.lib()
    assert lib.tusas_create(None, None, None) == pkg.EINVAL
    h = ctypes.c_void_p()
    assert lib.tusas_create(None, None, ctypes.byref(h)) == pkg.EINVAL
    assert lib.tusas_ndofs(None) == -1
    assert lib.tusas_last_error(None) == b"null handle"


def test_mesh_validation_rejects_bad_orders_before_gpu_work():
    """order must be 0/1 (Q1) or 2 (Q2); precond in 0..2."""
    import ctypes

    import paper_2006_16764_b300 as pkg
    from synth import Mesh, Params

    lib = pkg.lib()
    h = ctypes.c_void_p()
    for mesh, prm in [(Mesh(3, 4, 4, 4, 1.0, order=3), Params(precond=1)),
                      (Mesh(2, 4, 4, 0, 1.0, order=3), Params(precond=1)),
                      (Mesh(2, 4, 4, 0, 1.0, order=2), Params(precond=3))]:
        cm, cp = pkg.make_mesh(mesh), pkg.make_params(prm)
        assert lib.tusas_create(ctypes.byref(cm), ctypes.byref(cp), ctypes.byref(h)) == pkg.EINVAL
        assert not h.value


def test_device_bytes_cap_gives_enomem_before_gpu_work():
    """An allocation failure simulated by a size cap: tusas_create checks its vectors and
    Krylov basis against the cap before any CUDA call and returns TUSAS_ENOMEM."""
    import ctypes

    import paper_2006_16764_b300 as pkg
    from synth import Mesh, Params

    lib = pkg.lib()
    h = ctypes.c_void_p()
    mesh = Mesh(3, 32, 32, 32, 1.0)
    need = 8 * mesh.n_dofs * (11 + 2 * 30 + 1)  # vectors + GMRES(30) basis
    cm, cp = pkg.make_mesh(mesh), pkg.make_params(Params(precond=2))
    assert lib.tusas_set_device_bytes_cap(-1) == pkg.EINVAL
    try:
        pkg.set_device_bytes_cap(need - 8)
        assert lib.tusas_create(ctypes.byref(cm), ctypes.byref(cp), ctypes.byref(h)) == pkg.ENOMEM
        assert not h.value
        assert pkg.device_bytes() == 0
    finally:
        pkg.set_device_bytes_cap(0)
