"""FP64 CPU oracle of the fixed-mesh and moving-mesh (direct ALE) ADER-CWENO
steps -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package.  The product path (the CUDA
library under ``paper_1612_09335_gb300``) never imports, links or runs it, and
the two share no code; see ``oracle.cpp`` for the paper passages each
function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

EULER, MHD = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain g++ -O2)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P, D, I64, I = C.c_void_p, C.c_double, C.c_int64, C.c_int
            dp = C.POINTER(C.c_double)
            lp = C.POINTER(C.c_int64)
            ip = C.POINTER(C.c_int)
            cp = C.c_char_p
            L.orc_mesh_new.restype = P
            L.orc_mesh_new.argtypes = [I, I64, dp, I64, lp, dp, cp, I]
            L.orc_mesh_free.argtypes = [P]
            L.orc_mesh_geometry.argtypes = [P, dp, dp, dp, lp]
            L.orc_solver_new.restype = P
            L.orc_solver_new.argtypes = [P, I, I, dp, cp, I]
            L.orc_solver_free.argtypes = [P]
            L.orc_sizes.argtypes = [P, ip]
            L.orc_stencil.argtypes = [P, I64, lp, lp, cp, I]
            L.orc_reconstruct.argtypes = [P, dp, I64, lp, dp, dp, dp, dp, cp, I]
            L.orc_predictor.argtypes = [P, dp, D, I64, lp, dp, cp, I]
            L.orc_predictor_from_w.argtypes = [P, I64, dp, D, C.c_int, dp]
            L.orc_step.argtypes = [P, dp, D, I64, lp, dp, cp, I]
            L.orc_stable_dt.restype = D
            L.orc_stable_dt.argtypes = [P, dp, D]
            L.orc_physical_flux.argtypes = [I, I, dp, dp, I, dp]
            L.orc_max_speed_normal.restype = D
            L.orc_max_speed_normal.argtypes = [I, I, dp, dp, dp]
            L.orc_numerical_flux.argtypes = [I, I, dp, dp, dp, dp, dp]
            L.orc_abs_jacobian.argtypes = [I, D, dp, dp, dp]
            L.orc_max_speed.restype = D
            L.orc_max_speed.argtypes = [I, I, dp, dp]
            L.orc_gauss_rule.argtypes = [I, I, dp, dp]
            L.orc_simplex_integral.restype = D
            L.orc_simplex_integral.argtypes = [I, ip]
            L.orc_sigma.restype = D
            L.orc_sigma.argtypes = [P, dp]
            L.orc_monomials.argtypes = [P, ip]
            L.orc_st_nodes.argtypes = [P, dp]
            L.orc_face_points.argtypes = [P, I64, I, dp, dp, dp, dp]
            L.orc_face_points.restype = I
            L.orc_ale_step.argtypes = [P, dp, D, I, dp, dp, cp, I]
            L.orc_ale_predictor.argtypes = [P, dp, D, I, I64, dp, dp, cp, I]
            L.orc_ale_vertex_weights.argtypes = [P, dp]
            L.orc_st_normal.argtypes = [dp, dp, dp, dp, D, D, D, dp]
            L.orc_st_normal3.argtypes = [dp, dp, dp, dp, dp, dp, D, D, D, D, dp]
            L.orc_mesh_xyz.argtypes = [P, dp]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _l(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def default_params(dim: int = 2, pde: int = EULER, cfl: float | None = None, order: int = 3,
                   gamma: float | None = None, ch: float = 2.0, linear_weights: bool = False,
                   niter: int | None = None, positivity: bool = True, flux: int = 0) -> np.ndarray:
    """[eps, r, lambda0, lambda_s, gamma, c_h, cfl, picard iterations, linear_weights, positivity,
    flux (0 Rusanov, 1 Osher-type)]."""
    if gamma is None:
        gamma = 1.4 if pde == EULER else 5.0 / 3.0
    if cfl is None:
        cfl = 0.5 if dim == 2 else 1.0 / 3.0
    M = order - 1
    return np.array([1e-14, 4.0, 1e5, 1.0, gamma, ch, cfl, float(M + 1 if niter is None else niter),
                     1.0 if linear_weights else 0.0, 1.0 if positivity else 0.0, float(flux)])


class OracleMesh:
    def __init__(self, mesh):
        L = lib()
        self.dim = mesh.dim
        xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        cells = np.ascontiguousarray(mesh.cells, dtype=np.int64)
        per = None if mesh.period is None else np.ascontiguousarray(mesh.period, dtype=np.float64)
        err = C.create_string_buffer(256)
        self.h = L.orc_mesh_new(mesh.dim, xyz.shape[0], _d(xyz), cells.shape[0], _l(cells),
                                _d(per) if per is not None else None, err, 256)
        if not self.h:
            raise ValueError(err.value.decode())
        self.nc = cells.shape[0]
        self._keep = (xyz, cells, per)

    def xyz(self):
        """Current vertex positions (they change under ALE steps)."""
        out = np.zeros(self._keep[0].shape)
        lib().orc_mesh_xyz(self.h, _d(out))
        return out

    def geometry(self):
        L = lib()
        vol = np.zeros(self.nc)
        bary = np.zeros((self.nc, 3))
        h = np.zeros(self.nc)
        nbr = np.zeros((self.nc, self.dim + 1), dtype=np.int64)
        L.orc_mesh_geometry(self.h, _d(vol), _d(bary), _d(h), _l(nbr))
        return dict(vol=vol, bary=bary, h=h, nbr=nbr)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_mesh_free(self.h)
            self.h = None


class Oracle:
    """One (mesh, order, PDE, parameters) configuration of the oracle."""

    def __init__(self, mesh, order: int, pde: int = EULER, params=None):
        L = lib()
        self.mesh = mesh if isinstance(mesh, OracleMesh) else OracleMesh(mesh)
        self.dim = self.mesh.dim
        self.order = order
        self.pde = pde
        self.params = default_params(self.dim, pde, order=order) if params is None else np.asarray(params, float)
        err = C.create_string_buffer(256)
        self.h = L.orc_solver_new(self.mesh.h, order - 1, pde, _d(self.params), err, 256)
        if not self.h:
            raise ValueError(err.value.decode())
        s = np.zeros(5, dtype=np.int32)
        L.orc_sizes(self.h, _i(s))
        self.Mc, self.ne, self.L, self.L0, self.nu = (int(x) for x in s)
        self.nc = self.mesh.nc

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_solver_free(self.h)
            self.h = None

    @staticmethod
    def _ids(ids):
        if ids is None:
            return None, 0
        a = np.ascontiguousarray(ids, dtype=np.int64)
        return a, len(a)

    def stencil(self, cell: int):
        err = C.create_string_buffer(256)
        S0 = np.zeros(self.ne, dtype=np.int64)
        sec = np.zeros((self.dim + 1, self.dim), dtype=np.int64)
        if lib().orc_stencil(self.h, int(cell), _l(S0), _l(sec), err, 256) != 0:
            raise ValueError(err.value.decode())
        return S0, sec

    def reconstruct(self, Q, ids=None, want_popt=False, want_weights=False):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        a, n = self._ids(ids)
        cnt = n if a is not None else self.nc
        w = np.zeros((cnt, self.Mc, self.nu))
        popt = np.zeros_like(w) if want_popt else None
        om = np.zeros((cnt, self.dim + 2, self.nu)) if want_weights else None
        sg = np.zeros_like(om) if want_weights else None
        err = C.create_string_buffer(256)
        rc = lib().orc_reconstruct(self.h, _d(Q), n, _l(a) if a is not None else None, _d(w),
                                   _d(popt) if popt is not None else None,
                                   _d(om) if om is not None else None,
                                   _d(sg) if sg is not None else None, err, 256)
        if rc != 0:
            raise ValueError(err.value.decode())
        out = dict(w=w)
        if want_popt:
            out["popt"] = popt
        if want_weights:
            out["omega"] = om
            out["sigma"] = sg
        return out if (want_popt or want_weights) else w

    def predictor(self, Q, dt, ids=None):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        a, n = self._ids(ids)
        cnt = n if a is not None else self.nc
        q = np.zeros((cnt, self.L, self.nu))
        err = C.create_string_buffer(256)
        if lib().orc_predictor(self.h, _d(Q), float(dt), n, _l(a) if a is not None else None, _d(q), err,
                               256) != 0:
            raise ValueError(err.value.decode())
        return q

    def predictor_from_w(self, cell, wnodal, dt, galerkin=False):
        """Predictor of one cell from reconstruction values at the lattice
        nodes; galerkin=True solves the Galerkin system of Eq. (CGfinal)
        every iteration instead of using its closed form."""
        w = np.ascontiguousarray(wnodal, dtype=np.float64)
        q = np.zeros((self.L, self.nu))
        lib().orc_predictor_from_w(self.h, int(cell), _d(w), float(dt), int(bool(galerkin)), _d(q))
        return q

    def step(self, Q, dt, ids=None):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        a, n = self._ids(ids)
        cnt = n if a is not None else self.nc
        out = np.zeros((cnt, self.nu))
        err = C.create_string_buffer(256)
        if lib().orc_step(self.h, _d(Q), float(dt), n, _l(a) if a is not None else None, _d(out), err,
                          256) != 0:
            raise ValueError(err.value.decode())
        return out

    def stable_dt(self, Q, cfl=None):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        return lib().orc_stable_dt(self.h, _d(Q), float(self.params[6] if cfl is None else cfl))

    def run(self, Q, nsteps, dt=None, cfl=None):
        """nsteps full steps; dt None -> CFL time step each step."""
        Q = np.array(Q, dtype=np.float64)
        t = 0.0
        for _ in range(nsteps):
            h = self.stable_dt(Q, cfl) if dt is None else dt
            Q = self.step(Q, h)
            t += h
        return Q, t

    # ---- moving meshes (direct ALE, Secs. 2.2-2.4; 2D Euler, Rusanov)
    ALE_LAGRANGE, ALE_STILL = 1, 2

    def ale_step(self, Q, dt, mode=1):
        """One direct ALE step; returns (Q_new, xyz_new) and moves the
        oracle's mesh (stencils fixed)."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.zeros((self.nc, self.nu))
        xyz = np.zeros(self.mesh._keep[0].shape)
        err = C.create_string_buffer(256)
        if lib().orc_ale_step(self.h, _d(Q), float(dt), int(mode), _d(out), _d(xyz), err, 256) != 0:
            raise ValueError(err.value.decode())
        return out, xyz

    def ale_run(self, Q, nsteps, dt=None, mode=1, cfl=None):
        """nsteps ALE steps; dt None -> CFL time step on the current mesh."""
        Q = np.array(Q, dtype=np.float64)
        t = 0.0
        for _ in range(nsteps):
            h = self.stable_dt(Q, cfl) if dt is None else dt
            Q, _ = self.ale_step(Q, h, mode)
            t += h
        return Q, t

    def ale_predictor(self, Q, dt, cell, mode=1):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        q = np.zeros((self.L, self.nu))
        V = np.zeros((self.L, self.dim))
        err = C.create_string_buffer(256)
        if lib().orc_ale_predictor(self.h, _d(Q), float(dt), int(mode), int(cell), _d(q), _d(V), err, 256) != 0:
            raise ValueError(err.value.decode())
        return q, V

    def ale_vertex_weights(self):
        W = np.zeros((self.dim + 1, self.L))
        lib().orc_ale_vertex_weights(self.h, _d(W))
        return W

    def sigma(self, coef):
        c = np.ascontiguousarray(coef, dtype=np.float64)
        return lib().orc_sigma(self.h, _d(c))

    def monomials(self):
        e = np.zeros((self.Mc, 3), dtype=np.int32)
        lib().orc_monomials(self.h, _i(e))
        return e

    def st_nodes(self):
        x = np.zeros((self.L, 4))
        lib().orc_st_nodes(self.h, _d(x))
        return x

    def face_points(self, cell, k):
        M = self.order - 1
        npts = (M + 1) ** (self.dim - 1)
        pts = np.zeros((npts, 3))
        w = np.zeros(npts)
        n = np.zeros(3)
        area = np.zeros(1)
        lib().orc_face_points(self.h, int(cell), int(k), _d(pts), _d(w), _d(n), _d(area))
        return pts, w, n, float(area[0])


def physical_flux(pde, dim, q, m, params=None):
    p = default_params(dim, pde) if params is None else np.asarray(params, float)
    q = np.ascontiguousarray(q, dtype=np.float64)
    f = np.zeros(len(q))
    lib().orc_physical_flux(pde, dim, _d(p), _d(q), int(m), _d(f))
    return f


def numerical_flux(pde, dim, qm, qp, n, params=None):
    """Numerical normal flux at one point, unit normal n: Rusanov, Eq.
    (rusanov), or the Osher-type flux of Eq. (osher) when params[10] == 1."""
    p = default_params(dim, pde) if params is None else np.asarray(params, float)
    qm = np.ascontiguousarray(qm, dtype=np.float64)
    qp = np.ascontiguousarray(qp, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    g = np.zeros(len(qm))
    lib().orc_numerical_flux(pde, dim, _d(p), _d(qm), _d(qp), _d(n), _d(g))
    return g


def abs_jacobian(dim, q, n, gamma=1.4):
    """|A_n(q)| = R |Lambda| R^-1 of the Euler normal flux Jacobian."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    out = np.zeros((len(q), len(q)))
    lib().orc_abs_jacobian(dim, float(gamma), _d(q), _d(n), _d(out))
    return out


def max_speed_normal(pde, dim, q, n, params=None):
    p = default_params(dim, pde) if params is None else np.asarray(params, float)
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    return lib().orc_max_speed_normal(pde, dim, _d(p), _d(q), _d(n))


def max_speed(pde, dim, q, params=None):
    p = default_params(dim, pde) if params is None else np.asarray(params, float)
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().orc_max_speed(pde, dim, _d(p), _d(q))


def gauss_rule(kind, n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_rule(kind, n, _d(x), _d(w))
    return x, w


def simplex_integral(dim, e):
    a = np.ascontiguousarray(list(e) + [0] * (4 - len(e)), dtype=np.int32)
    return lib().orc_simplex_integral(dim, _i(a))


def st_normal(XA0, XB0, XA1, XB1, chi, tau, dt):
    """Space-time normal (x, y, t) of a moving 2D face at (chi, tau), Eq. (detChi)."""
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (XA0, XB0, XA1, XB1)]
    n = np.zeros(3)
    lib().orc_st_normal(_d(a[0]), _d(a[1]), _d(a[2]), _d(a[3]), float(chi), float(tau), float(dt), _d(n))
    return n


def st_normal3(A0, B0, C0, A1, B1, C1, chi1, chi2, tau, dt):
    """Space-time normal (x, y, z, t) of a moving triangle at (chi1, chi2, tau), Eq. (detChi)."""
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (A0, B0, C0, A1, B1, C1)]
    n = np.zeros(4)
    lib().orc_st_normal3(*[_d(x) for x in a], float(chi1), float(chi2), float(tau), float(dt), _d(n))
    return n
