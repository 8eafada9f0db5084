"""Thin ctypes binding of libcweno (include/cweno.h): argument marshalling only.

Every numerical step runs inside the CUDA library; this module converts numpy
arrays / CUDA tensors to pointers and error codes to exceptions.  It never
computes anything itself and has no fallback: if the library is missing it
raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import _build

EULER, MHD_GLM = 0, 1
FP64, FP32_MIXED = 0, 1
FLUX_RUSANOV, FLUX_OSHER, FLUX_RUSANOV_QF = 0, 1, 2
MOTION_FIXED, MOTION_LAGRANGE, MOTION_STILL = 0, 1, 2
OK, EINVAL, EDEGENERATE, ENOMEM, EBUSY, ENAN, ETIMEDOUT, ECUDA, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7, -8
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_ERROR = 0, 1, 2, 3


class CwenoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"cweno error {code}: {msg}")
        self.code = code


class cweno_params(C.Structure):
    _fields_ = [("eps", C.c_double), ("r", C.c_double), ("lambda0", C.c_double), ("lambda_s", C.c_double),
                ("gamma", C.c_double), ("c_h", C.c_double), ("cfl", C.c_double), ("picard_iters", C.c_int),
                ("linear_weights", C.c_int), ("positivity", C.c_int), ("flux", C.c_int),
                ("mesh_motion", C.c_int)]


class cweno_request(C.Structure):
    _fields_ = [("dim", C.c_int), ("nv", C.c_int64), ("xyz", C.POINTER(C.c_double)), ("nc", C.c_int64),
                ("cells", C.POINTER(C.c_int32)), ("period", C.POINTER(C.c_double)), ("order", C.c_int),
                ("pde", C.c_int), ("precision", C.c_int), ("Q0", C.POINTER(C.c_double)), ("cfl", C.c_double),
                ("nsteps", C.c_int)]


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) for every entry point of include/cweno.h
_P, _I, _I64, _D, _SZ = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_size_t
_DP, _IP, _I32P, _I64P, _U64P = (C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int64), C.POINTER(C.c_uint64))
SIGNATURES = [
    ("cweno_default_params", None, [C.POINTER(cweno_params), _I, _I]),
    ("cweno_last_error", C.c_char_p, []),
    ("cweno_nvars", _I, [_I, _I]),
    ("cweno_mesh_create", _I, [_I, _I64, _DP, _I64, _I32P, _DP, C.POINTER(_P)]),
    ("cweno_mesh_destroy", None, [_P]),
    ("cweno_mesh_info", _I, [_P, _I64P, _I64P, _I64P]),
    ("cweno_mesh_stencils", _I, [_P, _I, _I32P, _I32P]),
    ("cweno_solver_stencils", _I, [_P, _I32P, _I32P]),
    ("cweno_setup", _I, [_P, _I, _I, _I, C.POINTER(cweno_params), _P, C.POINTER(_P)]),
    ("cweno_solver_destroy", None, [_P]),
    ("cweno_solver_info", _I, [_P, _IP, _IP, _IP, _IP, _I64P, _I64P]),
    ("cweno_solver_footprint", _I, [_P, C.POINTER(_SZ)]),
    ("cweno_set_state", _I, [_P, _P, _I]),
    ("cweno_get_state", _I, [_P, _P, _I]),
    ("cweno_reconstruct", _I, [_P, _P, _I]),
    ("cweno_predictor", _I, [_P, _D, _P, _I]),
    ("cweno_stable_dt", _I, [_P, _D, _DP]),
    ("ader_cweno_step", _I, [_P, _D]),
    ("ader_cweno_run", _I, [_P, _I, _D]),
    ("cweno_sync", _I, [_P]),
    ("cweno_get_time", _I, [_P, _DP]),
    ("cweno_get_vertices", _I, [_P, _P, _I]),
    ("cweno_stream", _P, [_P]),
    ("cweno_profile_enable", _I, [_P, _I]),
    ("cweno_profile_read", _I, [_P, _DP, _I64P]),
    ("cweno_profile_read_stages", _I, [_P, _DP, _I64P, _I]),
    ("cweno_measure_fma_peak", _I, [_I, _DP, _DP]),
    ("cweno_stable_dt_noalloc", _I, [_I, _I, _I64, _P, _P, _D, _D, _D, _P, _P]),
    ("serve_create", _I, [_SZ, _I, _I, C.POINTER(_P)]),
    ("serve_submit", _I, [_P, C.POINTER(cweno_request), _U64P]),
    ("serve_poll", _I, [_P, C.c_uint64, _IP, _DP, _DP]),
    ("serve_drain", _I, [_P, _D]),
    ("serve_stats", _I, [_P, _U64P, _U64P, _U64P, _U64P, _DP]),
    ("serve_batch_stats", _I, [_P, _U64P, _U64P]),
    ("serve_destroy", None, [_P]),
]


def lib():
    """Load libcweno.so (built by paper_1612_09335_gb300.build())."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("CWENO_LIBRARY") or _build.LIB   # a variant build, for launch sweeps
            if not os.path.exists(path):
                raise RuntimeError("libcweno.so is not built; run paper_1612_09335_gb300.build() "
                                   "(the CUDA path has no fallback)")
            L = C.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise CwenoError(rc, lib().cweno_last_error().decode())


def _ptr(x):
    """(pointer, on_device) for a numpy array or a CUDA tensor (duck-typed)."""
    if hasattr(x, "data_ptr") and not x.is_contiguous():
        raise ValueError("tensor arguments must be contiguous")
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        return C.c_void_p(x.data_ptr()), 1
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr()), 0
    a = np.ascontiguousarray(x)
    return C.c_void_p(a.ctypes.data), 0


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------- same names
def cweno_default_params(dim: int, pde: int = EULER) -> cweno_params:
    p = cweno_params()
    lib().cweno_default_params(C.byref(p), dim, pde)
    return p


def cweno_nvars(dim: int, pde: int) -> int:
    return lib().cweno_nvars(dim, pde)


def cweno_mesh_create(dim: int, xyz, cells, period=None):
    xyz = _f64(xyz)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    per = None if period is None else _f64(period)
    h = C.c_void_p()
    _check(lib().cweno_mesh_create(dim, xyz.shape[0], xyz.ctypes.data_as(_DP), cells.shape[0],
                                   cells.ctypes.data_as(_I32P),
                                   per.ctypes.data_as(_DP) if per is not None else None, C.byref(h)))
    return h


def cweno_measure_fma_peak(fp64: bool) -> tuple[float, float]:
    """(TFLOP/s, ms) of the current device's FP32 (or FP64) FMA pipe, measured
    by an FMA-chain kernel timed with CUDA events (synchronous)."""
    t, ms = C.c_double(), C.c_double()
    _check(lib().cweno_measure_fma_peak(int(bool(fp64)), C.byref(t), C.byref(ms)))
    return t.value, ms.value


NOALLOC_MAX_CELLS = 65536 * 256


def _noalloc_check(dim: int, pde: int, Q_dev, h_dev, dt_dev) -> int:
    """The buffers cweno_stable_dt_noalloc reads and writes, checked before
    the call (the kernel reads ncells x nvars FP64 values of Q and ncells of
    h and writes one FP64 value to dt): CUDA, FP64, contiguous, of the right
    shape.  Returns ncells; raises CwenoError(EINVAL) otherwise."""
    import torch
    if dim not in (2, 3) or pde not in (EULER, MHD_GLM) or (dim == 3 and pde == MHD_GLM):
        raise CwenoError(EINVAL, "dim must be 2 or 3, pde EULER or MHD_GLM (MHD-GLM on 2D meshes only)")
    for name, t in (("Q", Q_dev), ("h", h_dev), ("dt", dt_dev)):
        if t.dtype != torch.float64:
            raise CwenoError(EINVAL, f"{name} must be float64, got {t.dtype}")
        if not t.is_cuda:
            raise CwenoError(EINVAL, f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise CwenoError(EINVAL, f"{name} must be contiguous")
    nv = cweno_nvars(dim, pde)
    if len(Q_dev.shape) != 2 or int(Q_dev.shape[1]) != nv:
        raise CwenoError(EINVAL, f"Q must have shape (ncells, {nv}), got {tuple(Q_dev.shape)}")
    n = int(Q_dev.shape[0])
    if h_dev.numel() < n:
        raise CwenoError(EINVAL, f"h has {h_dev.numel()} elements, fewer than the {n} cells of Q")
    if dt_dev.numel() < 1:
        raise CwenoError(EINVAL, "dt must hold one element")
    devs = {Q_dev.device, h_dev.device, dt_dev.device}
    if len(devs) != 1:
        raise CwenoError(EINVAL, "Q, h and dt must be on one device")
    return n


def cweno_stable_dt_noalloc(dim: int, pde: int, Q_dev, h_dev, gamma: float, c_h: float, cfl: float, dt_dev,
                            stream: int = 0):
    """CFL bound of a state held in the caller's device buffers, allocating
    nothing (Q_dev: ncells x nvars FP64 CUDA tensor, h_dev: ncells FP64, dt_dev:
    one FP64 element receiving the bound; asynchronous on `stream`).  The
    buffers are checked first (CwenoError EINVAL on a wrong dtype, device,
    layout or size), so the kernel never reads past them."""
    n = _noalloc_check(dim, pde, Q_dev, h_dev, dt_dev)
    _check(lib().cweno_stable_dt_noalloc(dim, pde, n, C.c_void_p(Q_dev.data_ptr()), C.c_void_p(h_dev.data_ptr()),
                                         float(gamma), float(c_h), float(cfl), C.c_void_p(dt_dev.data_ptr()),
                                         C.c_void_p(stream) if stream else None))


class Mesh:
    """Owned cweno_mesh handle."""

    def __init__(self, dim, xyz, cells, period=None):
        self.dim = dim
        self.h = cweno_mesh_create(dim, xyz, cells, period)
        self.nc = int(np.asarray(cells).shape[0])
        self.nv = int(np.asarray(xyz).shape[0])

    @classmethod
    def from_workload(cls, m):
        return cls(m.dim, m.xyz, m.cells, m.period)

    def info(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().cweno_mesh_info(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return dict(ncells=a.value, nfaces=b.value, nboundary=c.value)

    def stencils(self, order: int):
        # n_e = d M(M, d) cells (Eq. stencil); the library checks the order
        ne = self.dim * math.comb(max(order, 1) - 1 + self.dim, self.dim)
        S0 = np.zeros((self.nc, ne), dtype=np.int32)
        sec = np.zeros((self.nc, self.dim + 1, self.dim), dtype=np.int32)
        _check(lib().cweno_mesh_stencils(self.h, order, S0.ctypes.data_as(_I32P), sec.ctypes.data_as(_I32P)))
        return S0, sec

    def close(self):
        if getattr(self, "h", None):
            lib().cweno_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owned cweno_solver handle (cweno_setup)."""

    def __init__(self, mesh: Mesh, order: int, pde: int = EULER, precision: int = FP64, params=None,
                 stream=None, **overrides):
        p = cweno_default_params(mesh.dim, pde) if params is None else params
        for k, v in overrides.items():
            setattr(p, k, v)
        self.params = p
        h = C.c_void_p()
        _check(lib().cweno_setup(mesh.h, order, pde, precision, C.byref(p),
                                 C.c_void_p(stream) if stream else None, C.byref(h)))
        self.h = h
        self.mesh = mesh
        nv, mc, ne, lc = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        ncl, nf = C.c_int64(), C.c_int64()
        _check(lib().cweno_solver_info(h, C.byref(nv), C.byref(mc), C.byref(ne), C.byref(lc), C.byref(ncl),
                                       C.byref(nf)))
        self.nv, self.Mc, self.ne, self.L, self.nc, self.nf = nv.value, mc.value, ne.value, lc.value, ncl.value, nf.value
        self.order, self.pde, self.precision = order, pde, precision

    def footprint(self) -> int:
        b = C.c_size_t()
        _check(lib().cweno_solver_footprint(self.h, C.byref(b)))
        return b.value

    def stencils(self):
        """(S0 nc x n_e, sec nc x (d+1) x d): the stencils this solver uses."""
        S0 = np.zeros((self.nc, self.ne), dtype=np.int32)
        d = self.mesh.dim
        sec = np.zeros((self.nc, d + 1, d), dtype=np.int32)
        _check(lib().cweno_solver_stencils(self.h, S0.ctypes.data_as(_I32P), sec.ctypes.data_as(_I32P)))
        return S0, sec

    def set_state(self, Q):
        if not (hasattr(Q, "data_ptr") and getattr(Q, "is_cuda", False)):
            Q = _f64(Q)
        p, dev = _ptr(Q)
        _check(lib().cweno_set_state(self.h, p, dev))

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((self.nc, self.nv))
        p, dev = _ptr(out)
        _check(lib().cweno_get_state(self.h, p, dev))
        return out

    def reconstruct(self, out=None):
        if out is None:
            out = np.zeros((self.nc, self.Mc, self.nv))
        p, dev = _ptr(out)
        _check(lib().cweno_reconstruct(self.h, p, dev))
        return out

    def predictor(self, dt: float, out=None):
        if out is None:
            out = np.zeros((self.nc, self.L, self.nv))
        p, dev = _ptr(out)
        _check(lib().cweno_predictor(self.h, float(dt), p, dev))
        return out

    def stable_dt(self, cfl: float | None = None) -> float:
        d = C.c_double()
        _check(lib().cweno_stable_dt(self.h, float(self.params.cfl if cfl is None else cfl), C.byref(d)))
        return d.value

    def step(self, dt: float = 0.0):
        _check(lib().ader_cweno_step(self.h, float(dt)))

    def run(self, nsteps: int, dt: float = 0.0):
        _check(lib().ader_cweno_run(self.h, int(nsteps), float(dt)))

    def sync(self):
        _check(lib().cweno_sync(self.h))

    def time(self) -> float:
        t = C.c_double()
        _check(lib().cweno_get_time(self.h, C.byref(t)))
        return t.value

    def get_vertices(self, out=None):
        """Current vertex positions (moving meshes), nv x dim."""
        if out is None:
            out = np.zeros((self.mesh.nv, self.mesh.dim))
        p, dev = _ptr(out)
        _check(lib().cweno_get_vertices(self.h, p, dev))
        return out

    def stream(self) -> int:
        return lib().cweno_stream(self.h) or 0

    def profile(self, on: bool = True):
        _check(lib().cweno_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        ms = (C.c_double * 3)()
        n = (C.c_int64 * 3)()
        _check(lib().cweno_profile_read(self.h, ms, n))
        return list(ms), list(n)

    def profile_read_stages(self, nstages: int = 7):
        """Summed device ms and launch counts per stage since the last read
        (moving meshes: geometry + least squares, reconstruction, predictor,
        nodal solver, faces, update, CFL bound)."""
        ms = (C.c_double * nstages)()
        n = (C.c_int64 * nstages)()
        _check(lib().cweno_profile_read_stages(self.h, ms, n, int(nstages)))
        return list(ms), list(n)

    def close(self):
        if getattr(self, "h", None):
            lib().cweno_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owned cweno_server handle (serve_create / serve_submit / serve_poll)."""

    def __init__(self, mem_budget: int = 0, max_slots: int = 0, nworkers: int = 0):
        h = C.c_void_p()
        _check(lib().serve_create(int(mem_budget), int(max_slots), int(nworkers), C.byref(h)))
        self.h = h
        self._keep = {}
        self.errors = {}

    def submit(self, mesh, Q0, order: int, cfl: float, nsteps: int, pde: int = EULER,
               precision: int = FP32_MIXED) -> int:
        xyz = _f64(mesh.xyz)
        cells = np.ascontiguousarray(mesh.cells, dtype=np.int32)
        per = None if mesh.period is None else _f64(mesh.period)
        Q0 = _f64(Q0)
        r = cweno_request(mesh.dim, xyz.shape[0], xyz.ctypes.data_as(_DP), cells.shape[0],
                          cells.ctypes.data_as(_I32P), per.ctypes.data_as(_DP) if per is not None else None,
                          order, pde, precision, Q0.ctypes.data_as(_DP), float(cfl), int(nsteps))
        rid = C.c_uint64()
        _check(lib().serve_submit(self.h, C.byref(r), C.byref(rid)))
        self._keep[rid.value] = (cells.shape[0], Q0.shape[1])
        return rid.value

    def poll(self, rid: int, want_state: bool = True):
        st = C.c_int()
        lat = C.c_double()
        out = None
        nc, nv = self._keep.get(rid, (0, 0))
        if want_state and nc:
            out = np.zeros((nc, nv))
        _check(lib().serve_poll(self.h, C.c_uint64(rid), C.byref(st),
                                out.ctypes.data_as(_DP) if out is not None else None, C.byref(lat)))
        if st.value == REQ_ERROR:
            self.errors[rid] = lib().cweno_last_error().decode()
        if st.value != REQ_DONE:
            out = None
        return st.value, out, lat.value

    def drain(self, timeout_s: float = 600.0):
        _check(lib().serve_drain(self.h, float(timeout_s)))

    def stats(self):
        a, b, c, d = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        cu = C.c_double()
        _check(lib().serve_stats(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(cu)))
        t, ms = C.c_uint64(), C.c_uint64()
        _check(lib().serve_batch_stats(self.h, C.byref(t), C.byref(ms)))
        return dict(submitted=a.value, admitted=b.value, completed=c.value, peak_running=d.value,
                    cell_updates=cu.value, ticks=t.value, member_steps=ms.value)

    def close(self):
        if getattr(self, "h", None):
            lib().serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
