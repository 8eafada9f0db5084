"""Host-side checks of the C ABI (no GPU): the library builds, loads and
exports every entry point declared in include/cweno.h; mesh validation; the
stencils chosen by the library's setup equal the oracle's."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cw():
    import paper_1612_09335_gb300 as pkg
    pkg.build()
    from paper_1612_09335_gb300 import binding
    return binding


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "cweno.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b((?:cweno|ader|serve)_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(cw):
    L = cw.lib()
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(L, n), n
    bound = {s[0] for s in cw.SIGNATURES}
    assert set(names) == bound


def test_default_params_are_the_papers(cw):
    p = cw.cweno_default_params(2, cw.EULER)
    assert (p.eps, p.r, p.lambda0, p.lambda_s, p.gamma, p.cfl) == (1e-14, 4.0, 1e5, 1.0, 1.4, 0.5)
    p3 = cw.cweno_default_params(3, cw.EULER)
    assert abs(p3.cfl - 1 / 3) < 1e-15
    pm = cw.cweno_default_params(2, cw.MHD_GLM)
    assert abs(pm.gamma - 5 / 3) < 1e-15 and pm.c_h == 2.0
    assert cw.cweno_nvars(2, cw.EULER) == 4 and cw.cweno_nvars(3, cw.EULER) == 5 and cw.cweno_nvars(2, cw.MHD_GLM) == 9
    assert p.flux == cw.FLUX_RUSANOV and p.positivity == 1 and p.linear_weights == 0 and p.picard_iters == 0


def test_setup_rejects_unsupported_combinations_before_device_work(cw, wl):
    """Argument checks run before any device call (so they hold without a
    GPU): order range (both dimensions), order 5 outside the Euler
    equations, the Osher flux for MHD, an unknown flux."""
    m2 = cw.Mesh.from_workload(wl.tri_mesh(6))
    m3 = cw.Mesh.from_workload(wl.tet_mesh(3))
    cases = [(m2, 6, cw.EULER, {}), (m2, 1, cw.EULER, {}), (m3, 6, cw.EULER, {}), (m2, 5, cw.MHD_GLM, {}),
             (m2, 3, cw.MHD_GLM, {"flux": cw.FLUX_OSHER}), (m2, 3, cw.EULER, {"flux": 7})]
    for mesh, order, pde, kw in cases:
        with pytest.raises(cw.CwenoError) as e:
            cw.Solver(mesh, order, pde, **kw)
        assert e.value.code == cw.EINVAL, (order, pde, kw)


def test_moving_mesh_setup_rejects_unbuilt_combinations(cw, wl):
    """Moving meshes are built for Euler and the Rusanov flux, FP64 and
    FP32-mixed, orders 2..4; everything else is EINVAL before any device
    call."""
    m2 = cw.Mesh.from_workload(wl.tri_mesh(6))
    m3 = cw.Mesh.from_workload(wl.tet_mesh(3))
    cases = [(m3, 5, cw.EULER, cw.FP64, {}), (m3, 3, cw.EULER, cw.FP32_MIXED, {"flux": cw.FLUX_OSHER}),
             (m2, 3, cw.MHD_GLM, cw.FP64, {}), (m2, 5, cw.EULER, cw.FP64, {}),
             (m2, 5, cw.EULER, cw.FP32_MIXED, {}),
             (m2, 3, cw.EULER, cw.FP64, {"flux": cw.FLUX_OSHER}),
             (m2, 3, cw.EULER, cw.FP32_MIXED, {"flux": cw.FLUX_RUSANOV_QF})]
    for mesh, order, pde, prec, kw in cases:
        with pytest.raises(cw.CwenoError) as e:
            cw.Solver(mesh, order, pde, prec, mesh_motion=cw.MOTION_LAGRANGE, **kw)
        assert e.value.code == cw.EINVAL, (order, pde, prec, kw)
    with pytest.raises(cw.CwenoError) as e:
        cw.Solver(m2, 3, cw.EULER, cw.FP64, mesh_motion=7)
    assert e.value.code == cw.EINVAL


def test_mesh_validation_errors(cw, wl):
    m = wl.tri_mesh(4, jitter=0.1)
    bad = m.cells.copy()
    bad[3] = bad[3][[0, 2, 1]]  # clockwise cell
    with pytest.raises(cw.CwenoError) as e:
        cw.Mesh(2, m.xyz, bad, m.period)
    assert e.value.code == cw.EDEGENERATE
    bad = m.cells.copy()
    bad[0, 0] = 10 ** 6
    with pytest.raises(cw.CwenoError) as e:
        cw.Mesh(2, m.xyz, bad, m.period)
    assert e.value.code == cw.EINVAL
    with pytest.raises(cw.CwenoError) as e:
        cw.Mesh(4, m.xyz, m.cells, None)
    assert e.value.code == cw.EINVAL
    # a face shared by three cells
    cells = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], dtype=np.int32)
    xyz = np.array([[0, 0], [1, 0], [0, 1], [0.5, -1], [0.2, 2.0]])
    with pytest.raises(cw.CwenoError) as e:
        cw.Mesh(2, xyz, cells, None)
    assert e.value.code in (cw.EINVAL, cw.EDEGENERATE)


def test_mesh_counts(cw, wl):
    m = wl.tri_mesh(6, periodic=True)
    info = cw.Mesh.from_workload(m).info()
    assert info == dict(ncells=72, nfaces=108, nboundary=0)
    m = wl.tri_mesh(6, periodic=False)
    info = cw.Mesh.from_workload(m).info()
    assert info["nboundary"] == 24 and info["nfaces"] == (3 * 72 + 24) // 2
    m = wl.tet_mesh(3, periodic=True)
    info = cw.Mesh.from_workload(m).info()
    assert info == dict(ncells=162, nfaces=324, nboundary=0)


@pytest.mark.parametrize("case", [("tri", 10, True, 2), ("tri", 10, True, 3), ("tri", 10, True, 4),
                                  ("tri", 8, False, 3), ("tri", 8, False, 4), ("tet", 5, True, 2),
                                  ("tet", 5, True, 3), ("tet", 4, False, 3)])
def test_stencils_match_oracle(cw, orc, wl, case):
    kind, n, per, order = case
    m = wl.tri_mesh(n, periodic=per, jitter=0.2, seed=17) if kind == "tri" else \
        wl.tet_mesh(n, periodic=per, jitter=0.15, seed=17)
    S0, sec = cw.Mesh.from_workload(m).stencils(order)
    o = orc.Oracle(m, order)
    for c in range(0, m.nc, max(1, m.nc // 40)):
        s0o, seco = o.stencil(c)
        assert S0[c, 0] == c
        assert set(S0[c].tolist()) == set(s0o.tolist())
        for s in range(m.dim + 1):
            assert set(sec[c, s].tolist()) == set(seco[s].tolist()), (c, s)


def test_stencils_unjittered_ties_match_oracle(cw, orc, wl):
    """Exact distance ties (regular mesh) are broken the same way."""
    m = wl.tri_mesh(8, periodic=True, jitter=0.0)
    S0, sec = cw.Mesh.from_workload(m).stencils(3)
    o = orc.Oracle(m, 3)
    for c in range(0, m.nc, 5):
        s0o, seco = o.stencil(c)
        assert set(S0[c].tolist()) == set(s0o.tolist())
        for s in range(3):
            assert set(sec[c, s].tolist()) == set(seco[s].tolist())


def test_product_path_refuses_without_gpu_or_library(cw, wl):
    """Without a usable GPU, setup fails loudly (ECUDA); there is no CPU path."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    m = wl.tri_mesh(6)
    with pytest.raises(cw.CwenoError) as e:
        cw.Solver(cw.Mesh.from_workload(m), 3)
    assert e.value.code == cw.ECUDA


def test_predictor_zero_pattern_header_is_generated():
    """pred_pattern.h (the exact zero pattern of the predictor matrices that
    the kernels skip) is the output of its generator, which computes the
    entries in exact rational arithmetic."""
    import subprocess
    import sys
    csrc = os.path.join(ROOT, "paper_1612_09335_gb300", "csrc")
    out = subprocess.run([sys.executable, os.path.join(csrc, "gen_pred_pattern.py")], capture_output=True,
                         text=True, check=True).stdout
    assert out == open(os.path.join(csrc, "pred_pattern.h")).read()


def test_edge_case_meshes(cw, wl):
    """An empty mesh is refused (EINVAL); a mesh too small for the central
    stencil of the requested order is reported (EDEGENERATE, host setup);
    the smallest meshes that hold the stencil are accepted (8 bounded cells
    at second order: every cell has fewer than three neighbours)."""
    with pytest.raises(cw.CwenoError) as e:
        cw.Mesh(2, np.zeros((3, 2)), np.zeros((0, 3), np.int32), None)
    assert e.value.code == cw.EINVAL
    for n, per, ok_orders in ((3, True, (2, 3)), (3, False, (2, 3)), (2, False, (2,))):
        m = cw.Mesh.from_workload(wl.tri_mesh(n, periodic=per, jitter=0.0))
        for order in (2, 3, 4, 5):
            if order in ok_orders:
                S0, sec = m.stencils(order)
                assert S0.shape[0] == m.nc and (S0 >= 0).all()
            else:
                with pytest.raises(cw.CwenoError) as e:
                    m.stencils(order)
                assert e.value.code == cw.EDEGENERATE


class _FakeTensor:
    """Stands in for a tensor in the buffer checks of the allocation-free
    time-step call: the checks read only attributes, never memory."""

    def __init__(self, shape, dtype=None, is_cuda=True, contiguous=True, device="cuda:0"):
        import torch
        self.shape = tuple(shape)
        self.dtype = torch.float64 if dtype is None else dtype
        self.is_cuda = is_cuda
        self._contig = contiguous
        self.device = device

    def is_contiguous(self):
        return self._contig

    def numel(self):
        return int(np.prod(self.shape)) if self.shape else 1

    def data_ptr(self):
        raise AssertionError("the library must not be called when a buffer check fails")


def test_noalloc_binding_rejects_bad_buffers(cw):
    """The binding of cweno_stable_dt_noalloc checks every buffer before the
    call, so the kernel (which reads ncells x nvars FP64 values of Q and
    ncells of h) can never read past a caller's buffer: one rejection per
    check, and 3D MHD-GLM (not built) is refused like in cweno_setup."""
    import torch
    F = _FakeTensor
    good = dict(Q=F((100, 4)), h=F((100,)), dt=F((1,)))
    assert cw._noalloc_check(2, cw.EULER, good["Q"], good["h"], good["dt"]) == 100
    bad_cases = [
        (2, cw.EULER, F((100, 4), dtype=torch.float32), good["h"], good["dt"], "float64"),
        (2, cw.EULER, good["Q"], F((100,), dtype=torch.float32), good["dt"], "float64"),
        (2, cw.EULER, good["Q"], good["h"], F((1,), dtype=torch.float32), "float64"),
        (2, cw.EULER, F((100, 4), is_cuda=False), good["h"], good["dt"], "CUDA"),
        (2, cw.EULER, good["Q"], F((100,), is_cuda=False), good["dt"], "CUDA"),
        (2, cw.EULER, F((100, 4), contiguous=False), good["h"], good["dt"], "contiguous"),
        (2, cw.EULER, F((100, 3)), good["h"], good["dt"], "shape"),
        (3, cw.EULER, F((100, 4)), good["h"], good["dt"], "shape"),
        (2, cw.MHD_GLM, F((100, 4)), good["h"], good["dt"], "shape"),
        (2, cw.EULER, F((400,)), good["h"], good["dt"], "shape"),
        (2, cw.EULER, good["Q"], F((99,)), good["dt"], "fewer"),
        (2, cw.EULER, good["Q"], good["h"], F((0,)), "one element"),
        (2, cw.EULER, good["Q"], F((100,), device="cuda:1"), good["dt"], "one device"),
        (3, cw.MHD_GLM, F((100, 9)), good["h"], good["dt"], "2D meshes only"),
        (4, cw.EULER, F((100, 6)), good["h"], good["dt"], "dim"),
    ]
    for dim, pde, Q, h, dt, msg in bad_cases:
        with pytest.raises(cw.CwenoError) as e:
            cw.cweno_stable_dt_noalloc(dim, pde, Q, h, 1.4, 2.0, 0.5, dt)
        assert e.value.code == cw.EINVAL and msg in str(e.value), (dim, pde, msg, str(e.value))


def test_noalloc_entry_point_rejects_before_device_access(cw):
    """The C entry point itself refuses, before touching any pointer, the
    sizes beyond its static scratch and the pairings the solver does not
    build (3D MHD-GLM); no GPU is needed for either."""
    import ctypes as C
    L = cw.lib()
    fake = C.c_void_p(16)
    rc = L.cweno_stable_dt_noalloc(2, cw.EULER, cw.NOALLOC_MAX_CELLS + 1, fake, fake, 1.4, 2.0, 0.5, fake, None)
    assert rc == cw.EINVAL and "CWENO_NOALLOC_MAX_CELLS" in L.cweno_last_error().decode()
    rc = L.cweno_stable_dt_noalloc(3, cw.MHD_GLM, 1000, fake, fake, 5.0 / 3.0, 2.0, 0.5, fake, None)
    assert rc == cw.EINVAL and "2D meshes only" in L.cweno_last_error().decode()
