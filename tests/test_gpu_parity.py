"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  FP64 mode must agree to 1e-12 relative per variable,
||a_v - b_v||_inf / max(||b_v||_inf, 1e-6 max_u ||b_u||_inf) (a variable that
is identically zero, e.g. B_z or psi at t = 0, is measured against a
millionth of the state's scale); where the oracle's own response to one-ulp
input perturbations is larger (nonlinear weights at jumps, psi ~ div B
cancellations) the bound is eight times that response.  FP32-mixed mode is
held to the bounds stated below.  Mesh sizes span many thread blocks plus a
ragged tail."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EULER, MHD = 0, 1
TOL64 = 1e-12


@pytest.fixture(scope="module")
def cw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1612_09335_gb300 as pkg
    pkg.build()
    from paper_1612_09335_gb300 import binding
    return binding


def relerr(a, b, floor=1e-6):
    a = np.asarray(a).reshape(-1, np.asarray(a).shape[-1])
    b = np.asarray(b).reshape(-1, np.asarray(b).shape[-1])
    num = np.abs(a - b).max(axis=0)
    mag = np.abs(b).max(axis=0)
    den = np.maximum(np.maximum(mag, floor * mag.max()), 1e-300)
    return float((num / den).max())


def tolerance(name, fn, Q):
    """1e-12, or for discontinuous data the conditioning of the scheme: the
    nonlinear weights near a jump amplify a one-ulp change of the input by up
    to ~1e3, so the bound is 8x the oracle's own response to random relative
    input perturbations of 2^-52 (taken over three draws)."""
    base = fn(Q)
    rng = np.random.default_rng(123)
    worst = 0.0
    for _ in range(3):
        Qp = Q * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=Q.shape))
        worst = max(worst, relerr(fn(Qp), base))
    return max(TOL64, 8.0 * worst)


def case_inputs(wl, name):
    if name == "vortex2d":
        return wl.vortex_2d(16), EULER
    if name == "explosion2d":
        m = wl.tri_mesh(13, lo=(-1, -1), hi=(1, 1), periodic=False, jitter=0.2, seed=5)
        return (m, wl.explosion_averages(m, sub=6)), EULER
    if name == "wave3d":
        return wl.density_wave_3d(5), EULER
    if name == "explosion3d":
        m = wl.tet_mesh(5, lo=(-1, -1, -1), hi=(1, 1, 1), periodic=False, jitter=0.12, seed=5)
        return (m, wl.explosion_averages(m, sub=4)), EULER
    if name == "orszag":
        return wl.orszag_tang_2d(12), MHD
    raise KeyError(name)


CASES = [("vortex2d", 2), ("vortex2d", 3), ("vortex2d", 4), ("vortex2d", 5), ("explosion2d", 3),
         ("explosion2d", 4), ("explosion2d", 5), ("wave3d", 2), ("wave3d", 3), ("explosion3d", 3),
         ("orszag", 3), ("orszag", 4)]


def s_cfl(dim):
    return 0.5 if dim == 2 else 1.0 / 3.0


def make(cw, mesh, order, pde, prec, **kw):
    return cw.Solver(cw.Mesh.from_workload(mesh), order, pde, prec, **kw)


@pytest.mark.parametrize("name,order", CASES)
def test_reconstruct_fp64_matches_oracle(cw, orc, wl, name, order):
    (mesh, Q), pde = case_inputs(wl, name)
    s = make(cw, mesh, order, pde, cw.FP64)
    s.set_state(Q)
    w = s.reconstruct()
    o = orc.Oracle(mesh, order, pde)
    ref = o.reconstruct(Q)
    assert relerr(w, ref) < tolerance(name, o.reconstruct, Q)


@pytest.mark.parametrize("name,order", CASES)
def test_predictor_fp64_matches_oracle(cw, orc, wl, name, order):
    (mesh, Q), pde = case_inputs(wl, name)
    o = orc.Oracle(mesh, order, pde)
    dt = o.stable_dt(Q)
    s = make(cw, mesh, order, pde, cw.FP64)
    s.set_state(Q)
    q = s.predictor(dt)
    assert relerr(q, o.predictor(Q, dt)) < tolerance(name, lambda x: o.predictor(x, dt), Q)


@pytest.mark.parametrize("name,order", CASES)
def test_one_step_fp64_matches_oracle(cw, orc, wl, name, order):
    (mesh, Q), pde = case_inputs(wl, name)
    o = orc.Oracle(mesh, order, pde)
    dt = o.stable_dt(Q)
    s = make(cw, mesh, order, pde, cw.FP64)
    s.set_state(Q)
    s.step(dt)
    s.sync()
    Q1 = s.get_state()
    ref = o.step(Q, dt)
    assert relerr(Q1, ref) < tolerance(name, lambda x: o.step(x, dt), Q)
    # the increment itself (what the step computed) agrees to 1e-9 relative
    assert relerr(Q1 - Q, ref - Q) < 1e-9


@pytest.mark.parametrize("name,order", [("vortex2d", 3), ("wave3d", 3), ("orszag", 4), ("explosion2d", 4)])
def test_stable_dt_matches_oracle(cw, orc, wl, name, order):
    (mesh, Q), pde = case_inputs(wl, name)
    o = orc.Oracle(mesh, order, pde)
    s = make(cw, mesh, order, pde, cw.FP64)
    s.set_state(Q)
    assert abs(s.stable_dt(0.4) / o.stable_dt(Q, 0.4) - 1) < 1e-13


def test_config1_ten_steps_fp64(cw, orc, wl):
    """Periodic vortex, 32x32x2 triangles, P2, CFL 0.5, 10 steps: device time
    step (Eq. timestep) and the whole step chain against the oracle."""
    mesh, Q = wl.vortex_2d(32)
    o = orc.Oracle(mesh, 3)
    ref, tref = o.run(Q, 10)
    s = make(cw, mesh, 3, EULER, cw.FP64)
    s.set_state(Q)
    for _ in range(10):
        s.step(0.0)
    s.sync()
    assert abs(s.time() / tref - 1) < 1e-12
    assert relerr(s.get_state(), ref) < TOL64


def test_graph_run_equals_step_loop(cw, wl):
    mesh, Q = wl.vortex_2d(16)
    a = make(cw, mesh, 4, EULER, cw.FP32_MIXED)
    a.set_state(Q)
    for _ in range(7):
        a.step(0.0)
    a.sync()
    b = make(cw, mesh, 4, EULER, cw.FP32_MIXED)
    b.set_state(Q)
    b.run(7, 0.0)
    b.sync()
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.time() == b.time()


@pytest.mark.parametrize("prec", [0, 1])
def test_deterministic_bitwise(cw, wl, prec):
    mesh, Q = wl.vortex_2d(16)
    outs = []
    for _ in range(2):
        s = make(cw, mesh, 3, EULER, prec)
        s.set_state(Q)
        s.run(5)
        s.sync()
        outs.append(s.get_state())
    assert np.array_equal(outs[0], outs[1])


def test_state_roundtrip_and_device_pointers(cw, wl):
    import torch
    mesh, Q = wl.vortex_2d(16)
    s = make(cw, mesh, 3, EULER, cw.FP32_MIXED)
    s.set_state(Q)
    assert np.array_equal(s.get_state(), Q)
    Qd = torch.tensor(Q, device="cuda", dtype=torch.float64)
    torch.cuda.synchronize()
    s.set_state(Qd)
    out = torch.zeros_like(Qd)
    s.get_state(out)
    torch.cuda.synchronize()
    assert torch.equal(out, Qd)


@pytest.mark.parametrize("name,fp64", [("vortex2d", False), ("wave3d", True), ("orszag", False)])
def test_state_through_pinned_host_memory(cw, wl, name, fp64):
    """Page-locked host buffers are read and written in place by the state
    kernels; the result must equal the staged (pageable) path bit for bit,
    before and after a step."""
    import torch
    (mesh, Q), pde = case_inputs(wl, name)
    s = make(cw, mesh, 3, pde, cw.FP64 if fp64 else cw.FP32_MIXED)
    hin = torch.from_numpy(Q.copy()).pin_memory()
    s.set_state(hin)
    hout = torch.full(Q.shape, float("nan"), dtype=torch.float64).pin_memory()
    s.get_state(hout)
    assert np.array_equal(hout.numpy(), Q)
    s.step(0.0)
    a = s.get_state()
    s.get_state(hout)
    assert np.array_equal(hout.numpy(), a)
    s.set_state(Q)
    s.step(0.0)
    assert np.array_equal(s.get_state(), a)


@pytest.mark.parametrize("name,order", [("vortex2d", 3), ("vortex2d", 5), ("explosion2d", 4), ("wave3d", 3),
                                        ("wave3d", 5), ("orszag", 4)])
def test_conservation_both_modes(cw, wl, name, order):
    """Sum |T_i| Q_i is conserved on periodic meshes (and changes only by
    boundary fluxes otherwise): drift below 1e-12 relative in both modes."""
    (mesh, Q), pde = case_inputs(wl, name)
    if mesh.period is None:
        return conservation_with_boundary_flux(cw, wl, order)
    X = mesh.cell_vertices()
    E = X[:, 1:, :] - X[:, :1, :]
    vol = np.abs(np.linalg.det(E)) / math.factorial(mesh.dim)
    tot0 = vol @ Q
    for prec in (cw.FP64, cw.FP32_MIXED):
        s = make(cw, mesh, order, pde, prec)
        s.set_state(Q)
        s.run(20)
        s.sync()
        Q1 = s.get_state()
        tot = vol @ Q1
        scale = np.maximum(np.maximum(np.abs(tot0), vol @ np.abs(Q)), vol @ np.abs(Q1))
        scale = np.maximum(scale, 1e-6 * scale.max())
        assert np.all(np.abs(tot - tot0) <= 1e-12 * scale), (prec, tot - tot0)


def conservation_with_boundary_flux(cw, wl, order, nsteps=10):
    """Bounded (transmissive) mesh: sum |T_i| Q_i changes only by the boundary
    face integrals.  An explosion of radius 0.3 in [-1,1]^2 leaves a band of
    cells at the constant outer state q_out along the boundary for the first
    steps (checked), so every boundary face carries the flux of q_out
    (transmissive: q+ = q-, no Rusanov dissipation), and the expected change
    is -sum_n dt_n F(q_out) . sum_{boundary f} n_f |f|, computed here from the
    mesh and the time steps the solver reports."""
    mesh = wl.tri_mesh(40, lo=(-1, -1), hi=(1, 1), periodic=False, jitter=0.2, seed=5)
    Q = wl.explosion_averages(mesh, r0=0.3, sub=6)
    X = mesh.cell_vertices()
    vol = np.abs(np.linalg.det(X[:, 1:, :] - X[:, :1, :])) / 2.0
    # boundary edges (each belongs to one cell) with outward normals |f| n
    edges = {}
    for c in range(mesh.nc):
        for k in range(3):
            a, b = mesh.cells[c][(k + 1) % 3], mesh.cells[c][(k + 2) % 3]
            edges.setdefault((min(a, b), max(a, b)), []).append((c, a, b))
    nsum = np.zeros(2)
    bcells = set()
    for lst in edges.values():
        if len(lst) == 1:
            c, a, b = lst[0]
            t = mesh.xyz[b] - mesh.xyz[a]  # counter-clockwise cell: outward normal (t_y, -t_x)
            nsum += np.array([t[1], -t[0]])
            bcells.add(c)
    bcells = sorted(bcells)
    q_out = Q[bcells[0]].copy()
    assert np.all(Q[bcells] == q_out)
    gamma = 1.4
    rho, mx, my, E = q_out
    p = (gamma - 1) * (E - 0.5 * (mx * mx + my * my) / rho)
    Fx = np.array([mx, mx * mx / rho + p, mx * my / rho, mx / rho * (E + p)])
    Fy = np.array([my, my * mx / rho, my * my / rho + p, my / rho * (E + p)])
    Fn = Fx * nsum[0] + Fy * nsum[1]
    tot0 = vol @ Q
    for prec in (cw.FP64, cw.FP32_MIXED):
        s = make(cw, mesh, order, EULER, prec)
        s.set_state(Q)
        dts = []
        for _ in range(nsteps):
            dt = s.stable_dt()
            s.step(dt)
            dts.append(dt)
        s.sync()
        Q1 = s.get_state()
        # the premise: boundary cells still hold the outer state
        assert np.abs(Q1[bcells] - q_out).max() <= 1e-13 * np.abs(q_out).max(), prec
        expect = tot0 - sum(dts) * Fn
        tot = vol @ Q1
        scale = np.maximum(np.maximum(np.abs(tot0), vol @ np.abs(Q)), vol @ np.abs(Q1))
        scale = np.maximum(scale, 1e-6 * scale.max())
        assert np.all(np.abs(tot - expect) <= 1e-12 * scale), (prec, tot - expect)


@pytest.mark.parametrize("dim,pde,order", [(2, EULER, 4), (2, EULER, 5), (3, EULER, 3), (3, EULER, 5), (2, MHD, 4)])
def test_free_stream_both_modes(cw, wl, dim, pde, order):
    mesh = wl.tri_mesh(12, jitter=0.2, seed=3) if dim == 2 else wl.tet_mesh(5, jitter=0.15, seed=3)
    if pde == EULER:
        q = np.array([1.3, 0.4, -0.2, 0.1][:dim + 1] + [2.5])
    else:
        q = np.array([1.2, 0.3, -0.2, 0.1, 3.0, 0.5, -0.7, 0.2, 0.0])
    Q = np.tile(q, (mesh.nc, 1))
    # deviations from the cell average and the FP64 contraction of the face
    # sums keep a constant state constant to FP64 rounding in both modes
    # (error measured against the state's magnitude)
    for prec in (cw.FP64, cw.FP32_MIXED):
        s = make(cw, mesh, order, pde, prec)
        s.set_state(Q)
        s.run(3)
        s.sync()
        assert relerr(s.get_state(), Q, floor=1.0) < 1e-13


# FP32-mixed bounds against the FP64 oracle, one step from identical input,
# per variable relative L_inf with variables smaller than 1% of the state's
# scale measured at that scale (FP32 rounding is relative to the largest
# terms a variable is computed from).  Smooth Euler data: 2e-6;
# MHD-GLM: 3e-5 (psi and B_z come from cancellations in div B and the
# induction fluxes); discontinuous data: 1e-4 (weights near jumps amplify
# FP32 rounding of the indicators).
@pytest.mark.parametrize("name,order,tol", [("vortex2d", 3, 2e-6), ("vortex2d", 4, 2e-6), ("vortex2d", 5, 2e-6),
                                            ("explosion2d", 4, 1e-4), ("explosion2d", 5, 1e-4), ("wave3d", 3, 2e-6),
                                            ("orszag", 3, 3e-5), ("orszag", 4, 3e-5)])
def test_one_step_fp32_mixed_bounds(cw, orc, wl, name, order, tol):
    (mesh, Q), pde = case_inputs(wl, name)
    o = orc.Oracle(mesh, order, pde)
    dt = o.stable_dt(Q)
    s = make(cw, mesh, order, pde, cw.FP32_MIXED)
    s.set_state(Q)
    w = s.reconstruct()
    assert relerr(w, o.reconstruct(Q), floor=1e-2) < tol * 10
    s.step(dt)
    s.sync()
    Q1 = s.get_state()
    ref = o.step(Q, dt)
    per_var = [relerr(Q1[:, [v]], ref[:, [v]]) for v in range(Q.shape[1])]
    assert relerr(Q1, ref, floor=1e-2) < tol, per_var


def test_linear_weights_mode_on_gpu(cw, orc, wl):
    (mesh, Q), pde = case_inputs(wl, "explosion2d")
    prm = orc.default_params(2, EULER, order=4, linear_weights=True)
    o = orc.Oracle(mesh, 4, EULER, params=prm)
    s = make(cw, mesh, 4, EULER, cw.FP64, linear_weights=1)
    s.set_state(Q)
    assert relerr(s.reconstruct(), o.reconstruct(Q)) < TOL64


def test_nan_status_reported(cw, wl):
    """A state with negative pressure makes the next step report ENAN (host
    reads the status word; nothing traps on the device)."""
    mesh, Q = wl.vortex_2d(8)
    Q = Q.copy()
    Q[5, 3] = -1.0  # rho E < 0 -> negative pressure
    s = make(cw, mesh, 3, EULER, cw.FP64)
    s.set_state(Q)
    s.step(1e-4)
    with pytest.raises(cw.CwenoError) as e:
        s.sync()
    assert e.value.code == cw.ENAN


@pytest.mark.parametrize("prec", [0, 1])
def test_explosion_runs_admissible(cw, wl, prec):
    """Explosion, 96x96x2, P3: 60 steps stay finite and admissible in both
    precisions (positivity scaling on, the default)."""
    mesh, Q = wl.explosion_2d(96)
    s = make(cw, mesh, 4, EULER, prec)
    s.set_state(Q)
    s.run(60)
    s.sync()
    Q1 = s.get_state()
    p = 0.4 * (Q1[:, 3] - 0.5 * (Q1[:, 1] ** 2 + Q1[:, 2] ** 2) / Q1[:, 0])
    assert np.isfinite(Q1).all() and Q1[:, 0].min() > 0.1 and p.min() > 0.05


def test_positivity_off_is_the_papers_scheme(cw, orc, wl):
    (mesh, Q), pde = case_inputs(wl, "explosion2d")
    prm = orc.default_params(2, EULER, order=4, positivity=False)
    o = orc.Oracle(mesh, 4, EULER, params=prm)
    s = make(cw, mesh, 4, EULER, cw.FP64, positivity=0)
    s.set_state(Q)
    assert relerr(s.reconstruct(), o.reconstruct(Q)) < tolerance("explosion", o.reconstruct, Q)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,seed,order,r0,p_in", [(27, 1617, 2, 0.3786104969506505, 0.5165250010763427),
                                                 (165, 1689, 4, 0.3738107572554006, 0.55464529352432494)])
def test_explosions_from_serving_mix_stay_admissible(cw, wl, prec, n, seed, order, r0, p_in):
    """Two serving-mix requests that failed before the floor of 1e-3 and the
    predictor fallback: a P1 explosion (near-vacuum lattice node with finite
    momentum) and a P3 explosion (near-vacuum node with finite pressure, a
    sound speed 16x the cell average's).  50 steps at CFL 0.5 stay
    admissible in both precisions."""
    mesh = wl.tri_mesh(n, periodic=True, jitter=0.2, seed=seed)
    Q = wl.explosion_averages(mesh, r0=r0, centre=(0.5, 0.5), p_in=p_in, sub=4)
    s = make(cw, mesh, order, EULER, prec, cfl=0.5)
    s.set_state(Q)
    s.run(50)
    s.sync()  # raises on a non-admissible state
    Q1 = s.get_state()
    assert np.isfinite(Q1).all() and Q1[:, 0].min() > 0


def test_tiny_mesh_zero_steps_and_one_block(cw, orc, wl):
    """Edge cases: an 8-cell bounded mesh (second order; less than one thread
    block, boundary faces only around two cells) matches the oracle in FP64;
    zero steps leave the state untouched in both modes."""
    mesh = wl.tri_mesh(2, periodic=False, jitter=0.0)
    Q = wl.cell_averages(mesh, lambda x: wl.vortex(x, eps=2.0), n=4)
    o = orc.Oracle(mesh, 2, EULER)
    dt = o.stable_dt(Q)
    s = make(cw, mesh, 2, EULER, cw.FP64)
    s.set_state(Q)
    s.step(dt)
    s.sync()
    assert relerr(s.get_state(), o.step(Q, dt)) < TOL64
    for prec in (cw.FP64, cw.FP32_MIXED):
        s = make(cw, mesh, 2, EULER, prec)
        s.set_state(Q)
        s.run(0)
        s.sync()
        assert np.array_equal(s.get_state(), Q)


def test_fp32_pair_split_of_the_state(cw, wl):
    """FP32-mixed mode keeps each FP64 cell average as an FP32 pair (hi, lo).
    For a constant state the predictor is exactly the cell average at every
    node, returned as (double)hi + (double)lo, which must equal the FP64 value
    to 2^-46 relative (hi: 24 leading bits, lo: the rest rounded to FP32);
    exponents outside the integer-built range take the plain conversion."""
    mesh = wl.tri_mesh(8, jitter=0.2, seed=3)
    states = [
        [1.0, 0.0, -0.0, 2.5],
        [0.7, 1e-30, -2.5e-20, 3.3e15],
        [1.3, 1e-45, -7.77e30, 1e36],
        [2.0, 123456.789012345, -9.87654321e-7, 1.0 / 3.0],
        [1e-3, 1e-300, 5e-310, 2.0 ** -126],
    ]
    for q in states:
        q = np.array(q)
        Q = np.tile(q, (mesh.nc, 1))
        s = make(cw, mesh, 3, EULER, cw.FP32_MIXED)
        s.set_state(Q)
        out = s.predictor(1e-4)
        for v in range(4):
            got = out[..., v]
            assert np.all(got == got.flat[0]), (q[v], np.unique(got))
            g = float(got.flat[0])
            assert abs(g - q[v]) <= 2.0 ** -46 * abs(q[v]) + 1e-44, (q[v], g)
        s.close()


@pytest.mark.parametrize("kind,orders", [("tri_periodic", (2, 3, 4, 5)), ("tri_bounded", (2, 3, 4, 5)),
                                         ("tri_ties", (3, 4)), ("tet_periodic", (2, 3, 4, 5)),
                                         ("tet_bounded", (2, 3, 5))])
def test_device_stencil_search_equals_host_search(cw, wl, kind, orders):
    """cweno_setup finds the central stencils and sectors on the device; they
    must be the host search's (the rule the oracle's stencils are pinned to)
    cell for cell: jittered and unjittered (tie-breaking) meshes, periodic and
    bounded (dropped sectors), triangles and tetrahedra."""
    if kind == "tri_periodic":
        mesh = wl.tri_mesh(23, jitter=0.2, seed=17)
    elif kind == "tri_bounded":
        mesh = wl.tri_mesh(19, lo=(-1, -1), hi=(1, 1), periodic=False, jitter=0.2, seed=18)
    elif kind == "tri_ties":
        mesh = wl.tri_mesh(16, jitter=0.0)
    elif kind == "tet_periodic":
        mesh = wl.tet_mesh(6, jitter=0.15, seed=19)
    else:
        mesh = wl.tet_mesh(6, lo=(-1, -1, -1), hi=(1, 1, 1), periodic=False, jitter=0.12, seed=20)
    m = cw.Mesh.from_workload(mesh)
    for order in orders:
        S0h, sech = m.stencils(order)
        s = cw.Solver(m, order, cw.EULER, cw.FP32_MIXED)
        S0d, secd = s.stencils()
        s.close()
        assert np.array_equal(S0h, S0d), (kind, order)
        assert np.array_equal(sech, secd), (kind, order)
