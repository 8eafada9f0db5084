"""Full-size workloads, in the configuration bench.py times (device CFL time
step, FP32-mixed, plus FP64): one step on the whole mesh, compared with the
FP64 oracle on sampled cells that it computes one by one (each sampled cell
needs only its own and its face neighbours' reconstructions and predictors).

  explosion 2D P3  512x512x2 = 524,288 triangles, transmissive
  density wave 3D P2  64^3 x 6 = 1,572,864 tetrahedra, periodic
  Orszag-Tang MHD-GLM P3  724x724x2 = 1,048,352 triangles, periodic
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EULER, MHD = 0, 1


@pytest.fixture(scope="module")
def cw():
    import torch
    assert torch.cuda.is_available()
    import paper_1612_09335_gb300 as pkg
    pkg.build()
    from paper_1612_09335_gb300 import binding
    return binding


def relerr(a, b, floor=1e-6):
    num = np.abs(a - b).max(axis=0)
    mag = np.abs(b).max(axis=0)
    den = np.maximum(np.maximum(mag, floor * mag.max()), 1e-300)
    return float((num / den).max())


CONFIGS = {
    "explosion2d_p3": (lambda wl: wl.explosion_2d(512), 4, EULER, 1e-4),
    "densitywave3d_p2": (lambda wl: wl.density_wave_3d(64), 3, EULER, 2e-6),
    "orszagtang2d_p3": (lambda wl: wl.orszag_tang_2d(724), 4, MHD, 3e-5),
}


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_fullsize_one_step_sampled(cw, orc, wl, name):
    make, order, pde, tol32 = CONFIGS[name]
    mesh, Q = make(wl)
    rng = np.random.default_rng(11)
    ids = np.unique(np.concatenate([rng.choice(mesh.nc, 48, replace=False), [0, mesh.nc - 1]]))
    # cells touching the explosion front, where the nonlinear weights act
    if "explosion" in name:
        front = np.where((Q[:, 0] > 0.13) & (Q[:, 0] < 0.99))[0]
        ids = np.unique(np.concatenate([ids, rng.choice(front, 16, replace=False)]))
    o = orc.Oracle(mesh, order, pde)
    m = cw.Mesh.from_workload(mesh)
    for prec in (cw.FP64, cw.FP32_MIXED):
        s = cw.Solver(m, order, pde, prec)
        s.set_state(Q)
        dt = s.stable_dt()
        if prec == cw.FP64:
            assert abs(dt / o.stable_dt(Q) - 1) < 1e-13
        s.step(dt)
        s.sync()
        Q1 = s.get_state()[ids]
        ref = o.step(Q, dt, ids=ids)
        if prec == cw.FP64:
            # 1e-12, or 8x the oracle's own response to one-ulp input changes
            base = ref
            worst = 0.0
            for k in range(2):
                Qp = Q * (1.0 + 2.0 ** -52 * np.random.default_rng(k).choice([-1.0, 1.0], size=Q.shape))
                worst = max(worst, relerr(o.step(Qp, dt, ids=ids), base))
            assert relerr(Q1, ref) < max(1e-12, 8 * worst), (relerr(Q1, ref), worst)
        else:
            assert relerr(Q1, ref, floor=1e-2) < tol32
        s.close()
