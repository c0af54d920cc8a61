"""tusas-b300: Python binding of the C-ABI in include/tusas.h (argument marshalling only).

Every step of the hot path runs in the CUDA kernels of ``libtusas_b300.so``;
this module only converts torch tensors to pointers and checks return codes.
Import fails loudly (ImportError) when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtusas_b300.so")

OK, EINVAL, ECUDA, ENOMEM, ENOCONV, ENONFINITE = 0, -1, -2, -3, -4, -5
ERROR_NAMES = {EINVAL: "TUSAS_EINVAL", ECUDA: "TUSAS_ECUDA", ENOMEM: "TUSAS_ENOMEM",
               ENOCONV: "TUSAS_ENOCONV", ENONFINITE: "TUSAS_ENONFINITE"}

EXPORTS = ["tusas_create", "tusas_destroy", "tusas_set_stream", "tusas_set_params", "tusas_ndofs",
           "tusas_set_state", "tusas_set_history", "tusas_get_state", "tusas_time", "tusas_residual", "tusas_jvp",
           "tusas_jvp_fd", "tusas_jtvp", "tusas_jtvp_prev", "tusas_dFdp", "tusas_precond_setup",
           "tusas_precond_apply", "tusas_step", "tusas_dot", "tusas_last_error", "tusas_timers",
           "tusas_get_timers", "tusas_kernel_launches", "tusas_fma_peak", "tusas_forward", "tusas_adjoint", "tusas_solid_fraction",
           "tusas_set_device_bytes_cap", "tusas_device_bytes", "tusas_multidot_noalloc"]

TIMER_NAMES = ["residual", "residual_lin", "jv", "adjoint", "pc_apply", "pc_setup", "ortho"]


class CMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("order", ctypes.c_int)]


_PARAM_FIELDS = [
    ("model", ctypes.c_int),
    ("W0", ctypes.c_double), ("tau0", ctypes.c_double), ("eps4", ctypes.c_double), ("lam", ctypes.c_double),
    ("D", ctypes.c_double), ("k", ctypes.c_double),
    ("lT", ctypes.c_double), ("Vp", ctypes.c_double), ("zT", ctypes.c_double),
    ("theta", ctypes.c_double), ("phihat_form", ctypes.c_int),
    ("jat_normalised", ctypes.c_int), ("time_form", ctypes.c_int),
    ("jvp_mode", ctypes.c_int), ("precond", ctypes.c_int), ("smoother_fp32", ctypes.c_int),
    ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int), ("newton_maxit", ctypes.c_int),
    ("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double),
    ("eta0", ctypes.c_double), ("eta_min", ctypes.c_double), ("eta_max", ctypes.c_double),
    ("gamma", ctypes.c_double), ("omega", ctypes.c_double),
    ("mg_levels", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("coarse_degree", ctypes.c_int),
    ("linesearch_max", ctypes.c_int),
]


class CParams(ctypes.Structure):
    _fields_ = _PARAM_FIELDS


class CStats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("newton_its", ctypes.c_int), ("gmres_its", ctypes.c_int),
                ("linesearch_halvings", ctypes.c_int), ("residual_evals", ctypes.c_int),
                ("jv_evals", ctypes.c_int), ("fnorm0", ctypes.c_double), ("fnorm", ctypes.c_double),
                ("gmres_per_newton", ctypes.c_int * 32)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "gmres_per_newton"}
        d["gmres_per_newton"] = list(self.gmres_per_newton)[: self.newton_its]
        return d


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libtusas_b300.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, dp, i64 = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong
    sig = {
        "tusas_create": ([ctypes.POINTER(CMesh), ctypes.POINTER(CParams), ctypes.POINTER(vp)], ctypes.c_int),
        "tusas_destroy": ([vp], None),
        "tusas_set_stream": ([vp, vp], ctypes.c_int),
        "tusas_set_params": ([vp, ctypes.POINTER(CParams)], ctypes.c_int),
        "tusas_ndofs": ([vp], i64),
        "tusas_set_state": ([vp, dp, ctypes.c_double, ctypes.c_double], ctypes.c_int),
        "tusas_get_state": ([vp, dp], ctypes.c_int),
        "tusas_set_history": ([vp, dp], ctypes.c_int),
        "tusas_time": ([vp], ctypes.c_double),
        "tusas_residual": ([vp, dp, dp], ctypes.c_int),
        "tusas_jvp": ([vp, dp, dp, dp], ctypes.c_int),
        "tusas_jvp_fd": ([vp, dp, dp, dp], ctypes.c_int),
        "tusas_jtvp": ([vp, dp, dp, dp], ctypes.c_int),
        "tusas_jtvp_prev": ([vp, dp, dp, dp], ctypes.c_int),
        "tusas_dFdp": ([vp, dp, ctypes.c_int, dp], ctypes.c_int),
        "tusas_precond_setup": ([vp, dp], ctypes.c_int),
        "tusas_precond_apply": ([vp, dp, dp], ctypes.c_int),
        "tusas_step": ([vp, ctypes.POINTER(CStats)], ctypes.c_int),
        "tusas_dot": ([vp, dp, dp, i64, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "tusas_last_error": ([vp], ctypes.c_char_p),
        "tusas_timers": ([vp, ctypes.c_int], ctypes.c_int),
        "tusas_get_timers": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
        "tusas_kernel_launches": ([], i64),
        "tusas_multidot_noalloc": ([dp, i64, ctypes.c_int, dp, i64, ctypes.POINTER(ctypes.c_double), vp],
                                   ctypes.c_int),
        "tusas_forward": ([vp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                           ctypes.POINTER(CStats)], ctypes.c_int),
        "tusas_adjoint": ([vp, dp, dp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), dp,
                           ctypes.c_double, ctypes.POINTER(CStats)], ctypes.c_int),
        "tusas_fma_peak": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "tusas_solid_fraction": ([vp, dp, ctypes.POINTER(ctypes.c_double), dp], ctypes.c_int),
        "tusas_set_device_bytes_cap": ([i64], ctypes.c_int),
        "tusas_device_bytes": ([], i64),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def kernel_launches() -> int:
    """Kernels launched by the library in this process."""
    return int(lib().tusas_kernel_launches())


def fma_peak():
    """(FP64, FP32) FLOP/s of dependent FMA chains on the current device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = lib().tusas_fma_peak(ctypes.byref(a), ctypes.byref(b))
    if rc != OK:
        raise TusasError(rc, "tusas_fma_peak failed")
    return a.value, b.value


def set_device_bytes_cap(nbytes: int):
    """Cap the device bytes the library's handles may hold (0: no cap); past it allocations fail
    with TUSAS_ENOMEM as on a full device."""
    rc = lib().tusas_set_device_bytes_cap(int(nbytes))
    if rc != OK:
        raise TusasError(rc, "tusas_set_device_bytes_cap failed")


def device_bytes() -> int:
    """Device bytes held by the library's handles."""
    return int(lib().tusas_device_bytes())


NOALLOC_MAX_K = 32


def multidot_noalloc(X, k, y, n, ld=None, stream=None):
    """[X_j . y for j < k] without any device allocation (see tusas_multidot_noalloc).

    X: device tensor holding k vectors of stride ``ld`` (default n); y: device
    tensor of n doubles. Serialise overlapping calls: they share one scratch array.
    """
    out = (ctypes.c_double * max(int(k), 1))()
    raw = None if stream is None else ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = lib().tusas_multidot_noalloc(_ptr(X), int(n if ld is None else ld), int(k), _ptr(y), int(n), out, raw)
    if rc != OK:
        raise TusasError(rc, "tusas_multidot_noalloc failed")
    return [out[j] for j in range(int(k))]


class TusasError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def make_mesh(mesh) -> CMesh:
    return CMesh(int(mesh.dim), int(mesh.nx), int(mesh.ny), int(mesh.nz if mesh.dim == 3 else 0),
                 float(mesh.h), float(mesh.x0), float(mesh.y0), float(mesh.z0), int(getattr(mesh, "order", 1)))


def make_params(prm) -> CParams:
    c = CParams()
    for name, ty in _PARAM_FIELDS:
        setattr(c, name, (int if ty is ctypes.c_int else float)(getattr(prm, name)))
    return c


def _ptr(x):
    """Pointer of a torch tensor (CUDA or pinned CPU) or a contiguous numpy float64 array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be contiguous float64")
        return x.ctypes.data
    import torch

    if x.dtype != torch.float64 or not x.is_contiguous():
        raise ValueError("tensors must be contiguous float64")
    return x.data_ptr()


class Tusas:
    """One handle of the library: a structured box, parameters and a state U^n."""

    def __init__(self, mesh, params, stream=None):
        self.mesh = mesh
        self._lib = lib()
        self._cm = make_mesh(mesh)
        self._cp = make_params(params)
        h = ctypes.c_void_p()
        rc = self._lib.tusas_create(ctypes.byref(self._cm), ctypes.byref(self._cp), ctypes.byref(h))
        if rc != OK:
            raise TusasError(rc, "tusas_create failed")
        self._h = h
        self.n = int(self._lib.tusas_ndofs(self._h))
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tusas_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise TusasError(rc, self._lib.tusas_last_error(self._h).decode())
        return rc

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream (or its raw handle int)."""
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._check(self._lib.tusas_set_stream(self._h, ctypes.c_void_p(raw)))

    def set_params(self, params):
        self._cp = make_params(params)
        self._check(self._lib.tusas_set_params(self._h, ctypes.byref(self._cp)))

    def set_state(self, U, t, dt):
        self._check(self._lib.tusas_set_state(self._h, _ptr(U), float(t), float(dt)))

    def set_history(self, Unm1):
        self._check(self._lib.tusas_set_history(self._h, _ptr(Unm1)))

    def get_state(self, out):
        self._check(self._lib.tusas_get_state(self._h, _ptr(out)))
        return out

    @property
    def time(self):
        return float(self._lib.tusas_time(self._h))

    def residual(self, U, F):
        self._check(self._lib.tusas_residual(self._h, _ptr(U), _ptr(F)))
        return F

    def jvp(self, U, v, out):
        self._check(self._lib.tusas_jvp(self._h, _ptr(U), _ptr(v), _ptr(out)))
        return out

    def jvp_fd(self, U, v, out):
        self._check(self._lib.tusas_jvp_fd(self._h, _ptr(U), _ptr(v), _ptr(out)))
        return out

    def jtvp(self, U, w, out):
        self._check(self._lib.tusas_jtvp(self._h, _ptr(U), _ptr(w), _ptr(out)))
        return out

    def jtvp_prev(self, U, w, out):
        self._check(self._lib.tusas_jtvp_prev(self._h, _ptr(U), _ptr(w), _ptr(out)))
        return out

    def dFdp(self, U, out, which=0):
        self._check(self._lib.tusas_dFdp(self._h, _ptr(U), int(which), _ptr(out)))
        return out

    def precond_setup(self, U):
        self._check(self._lib.tusas_precond_setup(self._h, _ptr(U)))

    def precond_apply(self, r, z):
        self._check(self._lib.tusas_precond_apply(self._h, _ptr(r), _ptr(z)))
        return z

    def step(self, allow_noconv=False):
        st = CStats()
        rc = self._lib.tusas_step(self._h, ctypes.byref(st))
        if rc == ENOCONV and allow_noconv:
            return st.as_dict()
        self._check(rc)
        return st.as_dict()

    def forward(self, U0, t0, dt, nsteps, ckpt_every):
        """nsteps implicit steps from U0 recording checkpoints; returns summed step statistics."""
        st = CStats()
        self._check(self._lib.tusas_forward(self._h, _ptr(U0), float(t0), float(dt), int(nsteps),
                                            int(ckpt_every), ctypes.byref(st)))
        return st.as_dict()

    def adjoint(self, w, d0=None, g0=None, rtol=1e-10):
        """(dS/d eps4, dS/dU_0 . d0, stats) for S = w^T U_N of the last forward()."""
        ge, gd = ctypes.c_double(), ctypes.c_double()
        st = CStats()
        self._check(self._lib.tusas_adjoint(self._h, _ptr(w), _ptr(d0), ctypes.byref(ge), ctypes.byref(gd),
                                            _ptr(g0), float(rtol), ctypes.byref(st)))
        return ge.value, gd.value, st.as_dict()

    def solid_fraction(self, U):
        """S = int (1 + phi_h)/2 of the device state U (tusas_solid_fraction)."""
        S = ctypes.c_double()
        self._check(self._lib.tusas_solid_fraction(self._h, _ptr(U), ctypes.byref(S), None))
        return S.value

    def solid_fraction_weights(self, out):
        """Write dS/dU = [(1/2) int psi_i ; 0] into the device vector ``out``."""
        self._check(self._lib.tusas_solid_fraction(self._h, None, None, _ptr(out)))
        return out

    def timers(self, enable=True):
        self._check(self._lib.tusas_timers(self._h, int(enable)))

    def get_timers(self):
        """{class: (milliseconds, count)} of the enabled timers."""
        ms = (ctypes.c_double * len(TIMER_NAMES))()
        cnt = (ctypes.c_longlong * len(TIMER_NAMES))()
        self._check(self._lib.tusas_get_timers(self._h, ms, cnt))
        return {n: (ms[i], int(cnt[i])) for i, n in enumerate(TIMER_NAMES)}

    def dot(self, x, y, n=None):
        r = ctypes.c_double()
        n = self.n if n is None else int(n)
        self._check(self._lib.tusas_dot(self._h, _ptr(x), _ptr(y), n, ctypes.byref(r)))
        return r.value
