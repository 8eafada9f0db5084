"""cweno_stable_dt_noalloc: the CFL bound for callers that cannot allocate
device memory (inside a foreign memory pool, or with all device memory
reserved up front).  Its scratch is a static device array, so
the test checks, through the C ABI, that two calls in a row (different
states, different sizes) each give the bound the allocating entry point
cweno_stable_dt gives for the same state, to 1e-12 relative."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def char_sizes(mesh):
    """Incircle / insphere diameters 2 d |T| / sum |faces| (Eq. timestep)."""
    X = mesh.cell_vertices()
    d = mesh.dim
    vol = np.abs(np.linalg.det(X[:, 1:] - X[:, :1])) / math.factorial(d)
    surf = np.zeros(mesh.nc)
    for k in range(d + 1):
        P = X[:, [q for q in range(d + 1) if q != k]]
        if d == 2:
            surf += np.linalg.norm(P[:, 1] - P[:, 0], axis=1)
        else:
            surf += 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    return 2 * d * vol / surf


def test_noalloc_dt_matches_allocating_entry_point_twice():
    import torch
    assert torch.cuda.is_available()
    import paper_1612_09335_gb300 as pkg
    pkg.build()
    from paper_1612_09335_gb300 import binding as cw
    from paper_1612_09335_gb300 import workloads as wl

    cases = [(wl.vortex_2d(40), cw.EULER, 2), (wl.density_wave_3d(6), cw.EULER, 3),
             (wl.orszag_tang_2d(20), cw.MHD_GLM, 2)]
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for (mesh, Q), pde, dim in cases:
        s = cw.Solver(cw.Mesh.from_workload(mesh), 3, pde, cw.FP64)
        s.set_state(Q)
        cfl = 0.37
        ref = s.stable_dt(cfl)
        Qd = torch.tensor(Q, dtype=torch.float64, device="cuda")
        hd = torch.tensor(char_sizes(mesh), dtype=torch.float64, device="cuda")
        gamma = s.params.gamma
        for _ in range(2):
            dt_dev.fill_(-1.0)
            torch.cuda.synchronize()
            cw.cweno_stable_dt_noalloc(dim, pde, Qd, hd, gamma, s.params.c_h, cfl, dt_dev)
            torch.cuda.synchronize()
            got = float(dt_dev.item())
            assert abs(got / ref - 1) < 1e-12, (got, ref)


def test_noalloc_rejects_sizes_beyond_scratch():
    """Through the C ABI on a GPU process: sizes beyond the static scratch and
    3D MHD-GLM are refused before any device access (the pointers are never
    read)."""
    import ctypes as C
    import torch
    from paper_1612_09335_gb300 import binding as cw

    assert torch.cuda.is_available()
    L = cw.lib()
    fake = C.c_void_p(16)
    rc = L.cweno_stable_dt_noalloc(2, cw.EULER, cw.NOALLOC_MAX_CELLS + 1, fake, fake, 1.4, 2.0, 0.5, fake, None)
    assert rc == cw.EINVAL and "CWENO_NOALLOC_MAX_CELLS" in L.cweno_last_error().decode()
    rc = L.cweno_stable_dt_noalloc(3, cw.MHD_GLM, 1000, fake, fake, 5.0 / 3.0, 2.0, 0.5, fake, None)
    assert rc == cw.EINVAL and "2D meshes only" in L.cweno_last_error().decode()
