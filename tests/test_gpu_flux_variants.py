"""The other face fluxes on the GPU against the FP64 oracle: the Osher-type
flux of Eq. (osher) (Euler) and the quadrature-free Rusanov flux of the
fixed-mesh formulation (Euler and MHD-GLM).  Same one-step parity bounds as
the quadrature Rusanov path (FP64: 1e-12, or 8x the oracle's own response to
one-ulp input changes on discontinuous data; FP32-mixed: the stated
bounds), free-stream and conservation invariants, and the Osher flux's
defining advantage: a stationary contact stays sharp (no dissipation on the
entropy wave), where Rusanov smears it."""
import numpy as np
import pytest

from test_gpu_parity import EULER, MHD, case_inputs, make, relerr, tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cw():
    import torch
    assert torch.cuda.is_available()
    import paper_1612_09335_gb300 as pkg
    pkg.build()
    from paper_1612_09335_gb300 import binding
    return binding


OSHER, QF = 1, 2
CASES = [(OSHER, "vortex2d", 3), (OSHER, "vortex2d", 4), (OSHER, "vortex2d", 5), (OSHER, "explosion2d", 4),
         (OSHER, "explosion2d", 5), (OSHER, "wave3d", 2), (OSHER, "wave3d", 3), (OSHER, "explosion3d", 3),
         (QF, "vortex2d", 2), (QF, "vortex2d", 3), (QF, "vortex2d", 4), (QF, "vortex2d", 5),
         (QF, "explosion2d", 4), (QF, "explosion2d", 5), (QF, "wave3d", 2), (QF, "wave3d", 3),
         (QF, "explosion3d", 3), (QF, "orszag", 3), (QF, "orszag", 4)]


@pytest.mark.parametrize("flux,name,order", CASES)
def test_one_step_fp64_matches_oracle(cw, orc, wl, flux, name, order):
    (mesh, Q), pde = case_inputs(wl, name)
    prm = orc.default_params(mesh.dim, pde, order=order, flux=flux)
    o = orc.Oracle(mesh, order, pde, params=prm)
    dt = o.stable_dt(Q)
    s = make(cw, mesh, order, pde, cw.FP64, flux=flux)
    s.set_state(Q)
    s.step(dt)
    s.sync()
    got = s.get_state()
    tol = tolerance(name, lambda q: o.step(q, dt), Q)
    assert relerr(got, o.step(Q, dt)) < tol


@pytest.mark.parametrize("flux,name,order,tol", [(OSHER, "vortex2d", 4, 2e-6), (OSHER, "vortex2d", 5, 2e-6),
                                                 (OSHER, "explosion2d", 4, 1e-4), (OSHER, "wave3d", 3, 2e-6),
                                                 (QF, "vortex2d", 4, 2e-6), (QF, "explosion2d", 4, 1e-4),
                                                 (QF, "wave3d", 3, 2e-6), (QF, "orszag", 4, 3e-5)])
def test_one_step_fp32_mixed_bounds(cw, orc, wl, flux, name, order, tol):
    (mesh, Q), pde = case_inputs(wl, name)
    o = orc.Oracle(mesh, order, pde, params=orc.default_params(mesh.dim, pde, order=order, flux=flux))
    dt = o.stable_dt(Q)
    s = make(cw, mesh, order, pde, cw.FP32_MIXED, flux=flux)
    s.set_state(Q)
    s.step(dt)
    s.sync()
    assert relerr(s.get_state(), o.step(Q, dt), floor=1e-2) < tol


@pytest.mark.parametrize("flux,dim,order", [(OSHER, 2, 4), (OSHER, 3, 3), (QF, 2, 4), (QF, 3, 3)])
def test_free_stream_and_conservation(cw, wl, flux, dim, order):
    mesh = wl.tri_mesh(12, jitter=0.2, seed=3) if dim == 2 else wl.tet_mesh(5, jitter=0.15, seed=3)
    q = np.array([1.3, 0.4, -0.2, 0.1][:dim + 1] + [2.5])
    for prec in (cw.FP64, cw.FP32_MIXED):
        s = make(cw, mesh, order, EULER, prec, flux=flux)
        s.set_state(np.tile(q, (mesh.nc, 1)))
        s.run(3)
        s.sync()
        assert relerr(s.get_state(), np.tile(q, (mesh.nc, 1)), floor=1.0) < 1e-13
    (m2, Q), _ = case_inputs(wl, "vortex2d") if dim == 2 else case_inputs(wl, "wave3d")
    X = m2.cell_vertices()
    vol = np.abs(np.linalg.det(X[:, 1:] - X[:, :1])) / (2 if dim == 2 else 6)
    for prec in (cw.FP64, cw.FP32_MIXED):
        s = make(cw, m2, order, EULER, prec, flux=flux)
        s.set_state(Q)
        s.run(10)
        s.sync()
        Q1 = s.get_state()
        tot0, tot = vol @ Q, vol @ Q1
        scale = np.maximum(np.maximum(np.abs(tot0), vol @ np.abs(Q)), 1e-6)
        assert np.all(np.abs(tot - tot0) <= 1e-12 * scale)


def test_osher_keeps_stationary_contact_sharp(cw, wl):
    """Density jump at rest with equal pressure (an exact steady solution):
    the Osher flux has no dissipation on the entropy wave, so the cell
    averages do not move (to rounding); Rusanov diffuses the jump."""
    mesh = wl.tri_mesh(24, lo=(-1, -1), hi=(1, 1), periodic=False, jitter=0.0, seed=1)
    X = mesh.cell_vertices()
    xc = X.mean(axis=1)[:, 0]
    # the jump sits on grid lines (x = 0), so every cell is on one side
    rho = np.where(xc < 0.0, 1.0, 0.125)
    Q = np.column_stack([rho, np.zeros_like(rho), np.zeros_like(rho), np.full_like(rho, 1.0 / 0.4)])
    out = {}
    for flux in (cw.FLUX_OSHER, cw.FLUX_RUSANOV):
        s = make(cw, mesh, 3, EULER, cw.FP64, flux=flux)
        s.set_state(Q)
        s.run(10)
        s.sync()
        out[flux] = np.abs(s.get_state() - Q).max()
    assert out[cw.FLUX_OSHER] < 1e-12, out
    assert out[cw.FLUX_RUSANOV] > 1e-3, out
