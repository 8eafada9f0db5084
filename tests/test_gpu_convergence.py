"""Design-order convergence on the isentropic vortex of Sec. 4.1 (Eqs.
ShuVortIC, ShuVortDelta): the paper's domain [0,10]^2, periodic, epsilon = 5,
v_c = (1,1), t_f = 1, CFL 0.5, exact solution the translated initial data.
Errors are L1 norms of the density cell averages against the exact cell
averages on 64^2, 128^2, 256^2 x 2 jittered triangles.

* The linear scheme (omega = lambda) must show the design order M+1 on the
  finest pair (this pins reconstruction, predictor, fluxes and update).
* With the paper's weights (eps = 1e-14, r = 4) the weight of P_0 drops next
  to the vortex's critical points; measured: P2 2.78 -> 3.14, P3 2.74 -> 3.09
  (and 2.95 at 512^2), P4 2.55 -> 3.15 (still rising; the linear P4 scheme:
  4.85 -> 4.88).  Required: P2 >= 2.7, P3 >= 2.9, P4 >= 3.0.
* FP32-mixed must not lower the order: its rate matches the FP64 rate within
  0.1 on every pair whose finer FP64 error is above 1e-4 (two orders above
  the FP32 floor of about 1e-6 here)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cw():
    import torch
    assert torch.cuda.is_available()
    import paper_1612_09335_gb300 as pkg
    pkg.build()
    from paper_1612_09335_gb300 import binding
    return binding


def vortex(wl, x, t=0.0):
    return wl.vortex(x, t=t, eps=5.0, centre=(5.0, 5.0), scale=1.0, L=(10.0, 10.0))


def l1_error(cw, wl, n, order, prec, tf=1.0, linear=0):
    mesh = wl.tri_mesh(n, lo=(0.0, 0.0), hi=(10.0, 10.0), periodic=True, jitter=0.2, seed=1234)
    Q0 = wl.cell_averages(mesh, lambda x: vortex(wl, x), n=6)
    s = cw.Solver(cw.Mesh.from_workload(mesh), order, cw.EULER, prec, linear_weights=linear)
    s.set_state(Q0)
    t = 0.0
    while t < tf - 1e-14:
        dt = min(s.stable_dt(), tf - t)
        s.step(dt)
        t += dt
    s.sync()
    Q = s.get_state()
    ex = wl.cell_averages(mesh, lambda x: vortex(wl, x, t=tf), n=6)
    X = mesh.cell_vertices()
    vol = np.abs(np.linalg.det(X[:, 1:] - X[:, :1])) / 2
    return float(vol @ np.abs(Q[:, 0] - ex[:, 0]))


@pytest.mark.parametrize("order", [3, 4, 5])
def test_vortex_design_order_fp64_and_fp32(cw, wl, order):
    ns = (64, 128, 256)
    runs = {(p, lin): [l1_error(cw, wl, n, order, p, linear=lin) for n in ns]
            for p in (cw.FP64, cw.FP32_MIXED) for lin in (0, 1)}
    rates = {k: [math.log(e[j] / e[j + 1], 2) for j in range(len(ns) - 1)] for k, e in runs.items()}
    print("order", order, "errors", runs, "rates", rates)
    assert rates[(cw.FP64, 1)][-1] > order - 0.3, (runs, rates)
    assert rates[(cw.FP64, 0)][-1] > {3: 2.7, 4: 2.9, 5: 3.0}[order], (runs, rates)
    checked = 0
    for lin in (0, 1):
        for j in range(len(ns) - 1):
            if runs[(cw.FP64, lin)][j + 1] > 1e-4:
                assert abs(rates[(cw.FP32_MIXED, lin)][j] - rates[(cw.FP64, lin)][j]) < 0.1, (runs, rates)
                checked += 1
    assert checked >= 2
