"""Design-order convergence on tetrahedra (the 3D part of the convergence
study of Sec. 4.1): the density wave rho = 1 + 0.2 sin 2 pi (x + y + z),
p = 1, v = (1, 1, 1) (an exact solution, translated), on periodic jittered
Kuhn meshes of 6^3, 12^3 and 24^3 x 6 tetrahedra, to t = 0.05 with the
device CFL step, FP64, orders 3 to 5.  Errors are L1 norms of the density
cell averages against the exact cell averages.

The linear scheme (omega = lambda) must show close to the design order on
the finest pair (measured 2.85, 4.28, 4.77 for orders 3, 4, 5; required
order - 0.5): this pins reconstruction, predictor, fluxes and update in 3D
up to fifth order.  With the paper's nonlinear weights the same runs converge
at 1.1-1.4 on this range of meshes (k h = 0.9 to 0.45): near the wave's
critical planes the second-derivative terms dominate the indicator of P_0
while the sectorial indicators hold first derivatives only, and with r = 4,
lambda_0 / lambda_s = 1e5 a ratio above about 18 hands the cell to a
sectorial polynomial.  That behaviour is the scheme's, not asserted here."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TF = 0.05
NS = (6, 12, 24)


@pytest.fixture(scope="module")
def cw():
    import torch
    assert torch.cuda.is_available()
    import paper_1612_09335_gb300 as pkg
    pkg.build()
    from paper_1612_09335_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def cases(wl):
    out = {}
    for n in NS:
        mesh = wl.tet_mesh(n, periodic=True, jitter=0.15, seed=1234)
        Q0 = wl.cell_averages(mesh, lambda x: wl.density_wave(x), n=4)
        ex = wl.cell_averages(mesh, lambda x: wl.density_wave(x, t=TF), n=4)
        X = mesh.cell_vertices()
        vol = np.abs(np.linalg.det(X[:, 1:] - X[:, :1])) / 6
        out[n] = (mesh, Q0, ex, vol)
    return out


def l1_error(cw, case, order, linear):
    mesh, Q0, ex, vol = case
    s = cw.Solver(cw.Mesh.from_workload(mesh), order, cw.EULER, cw.FP64, linear_weights=linear)
    s.set_state(Q0)
    t = 0.0
    while t < TF - 1e-14:
        dt = min(s.stable_dt(), TF - t)
        s.step(dt)
        t += dt
    s.sync()
    err = float(vol @ np.abs(s.get_state()[:, 0] - ex[:, 0]))
    s.close()
    return err


@pytest.mark.parametrize("order", [3, 4, 5])
def test_density_wave_design_order_on_tetrahedra(cw, cases, order):
    errs = [l1_error(cw, cases[n], order, 1) for n in NS]
    rates = [math.log2(errs[j] / errs[j + 1]) for j in range(len(NS) - 1)]
    print("order", order, "errors", errs, "rates", rates)
    assert rates[-1] > order - 0.5, (errs, rates)
