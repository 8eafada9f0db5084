"""Pins of the oracle's moving-mesh (direct ALE) step, Secs. 2.2-2.4, against
facts fixed by the mathematics rather than by the oracle itself:

* V = 0 turns the ALE machinery (Galerkin predictor with nodal H, space-time
  faces, volume-weighted update) into the Eulerian scheme, whose oracle is
  pinned separately;
* Galilean invariance: a Lagrangian step of a density wave translating with
  u = (1, 1) gives, in exact arithmetic, the same densities as the Eulerian
  step of the co-moving (stationary) wave on the same mesh;
* constant states stay constant under any mesh motion (the GCL of Eq. gcl),
  and with V = v the mesh translates with the flow;
* the space-time normal of Eq. (detChi) closes every moving triangle:
  the lateral integrals of n~ equal (0, 0, |T^n| - |T^{n+1}|), areas by the
  shoelace formula;
* the vertex-velocity weights of Eq. (NodesVel) integrate polynomials in tau
  exactly;
* the moving-element predictor of an affine density with constant velocity
  and pressure is constant in tau in the co-moving reference frame (H = 0).
"""
import math

import numpy as np
import pytest

EULER = 0


@pytest.fixture(scope="module")
def orc():
    import oracle
    return oracle


@pytest.fixture(scope="module")
def wl():
    from paper_1612_09335_gb300 import workloads
    return workloads


def _wave(wl, x, u):
    s = x[:, 0] + x[:, 1]
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * s)
    return wl.euler_conserved(rho, np.full((2, len(rho)), u), np.ones_like(rho), 1.4)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_ale_still_mesh_is_the_eulerian_step(orc, wl, order):
    mesh, Q = wl.vortex_2d(8)
    dt = orc.Oracle(mesh, order).stable_dt(Q)
    a = orc.Oracle(mesh, order).step(Q, dt)
    b, xyz = orc.Oracle(mesh, order).ale_step(Q, dt, mode=2)
    assert np.array_equal(xyz, mesh.xyz)
    # the Galerkin solve of Eq. (CGfinal) rounds at cond(K_tau^1) ~ 1.5e4 (M = 3)
    assert np.abs(a - b).max() / np.abs(a).max() < 1e-12


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("linear", [False, True])
def test_ale_galilean_invariance(orc, wl, order, linear):
    mesh, _ = wl.density_wave_2d(12)
    Qm = wl.cell_averages(mesh, lambda x: _wave(wl, x, 1.0), n=6)
    Qs = wl.cell_averages(mesh, lambda x: _wave(wl, x, 0.0), n=6)
    prm = orc.default_params(2, EULER, order=order, linear_weights=linear)
    dt = 0.004
    a, xyz = orc.Oracle(mesh, order, params=prm).ale_step(Qm, dt, mode=1)
    b = orc.Oracle(mesh, order, params=prm).step(Qs, dt)
    assert np.abs(xyz - mesh.xyz - dt).max() < 1e-15
    assert np.abs(a[:, 0] - b[:, 0]).max() < 1e-12
    assert np.abs((a[:, 1] - a[:, 0]) - b[:, 1]).max() < 1e-12
    assert np.abs(a[:, 0] - Qm[:, 0]).max() > 1e-4  # the step did change the densities


@pytest.mark.parametrize("order", [2, 4])
def test_ale_constant_state_and_translation(orc, wl, order):
    mesh, _ = wl.vortex_2d(8)
    q = np.array([1.3, 0.39, -0.26, 3.1])
    Q = np.tile(q, (mesh.nc, 1))
    o = orc.Oracle(mesh, order)
    x0 = mesh.xyz.copy()
    for _ in range(2):
        Q, xyz = o.ale_step(Q, 0.01, mode=1)
    # order 4: the Galerkin solve (cond 1.5e4) rounds the nodal states at ~1e-13
    assert np.abs(Q - q).max() < (1e-14 if order == 2 else 5e-13)
    assert np.abs(xyz - x0 - 0.02 * q[1:3] / q[0]).max() < 1e-14


def _shoelace(P):
    x, y = P[:, 0], P[:, 1]
    return 0.5 * (x[0] * (y[1] - y[2]) + x[1] * (y[2] - y[0]) + x[2] * (y[0] - y[1]))


def test_space_time_normals_close_a_moving_triangle(orc):
    rng = np.random.default_rng(7)
    gx, gw = orc.gauss_rule(0, 2)  # the time part of n~ is bilinear: 2x2 points are exact
    for _ in range(20):
        P0 = np.array([[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]]) + 0.1 * rng.standard_normal((3, 2))
        P1 = P0 + 0.2 * rng.standard_normal((3, 2))
        dt = rng.uniform(0.01, 0.5)
        tot = np.zeros(3)
        c0 = P0.mean(axis=0)
        for k in range(3):
            A, B = (k + 1) % 3, (k + 2) % 3
            n00 = orc.st_normal(P0[A], P0[B], P1[A], P1[B], 0.0, 0.0, dt)
            sgn = 1.0 if n00[:2] @ (P0[A] - c0) > 0 else -1.0
            for a in range(2):
                for t in range(2):
                    tot += sgn * gw[a] * gw[t] * orc.st_normal(P0[A], P0[B], P1[A], P1[B], gx[a], gx[t], dt)
        assert abs(tot[0]) < 1e-13 and abs(tot[1]) < 1e-13
        assert abs(tot[2] - (_shoelace(P0) - _shoelace(P1))) < 1e-13


def test_space_time_normal_still_and_translating_face(orc):
    A0, B0 = np.array([0.2, 0.1]), np.array([0.7, 0.5])
    e = B0 - A0
    n = orc.st_normal(A0, B0, A0, B0, 0.3, 0.6, 0.25)
    assert np.allclose(n, [0.25 * e[1], -0.25 * e[0], 0.0], atol=1e-16)
    V = np.array([0.4, -1.1])
    dt = 0.3
    n = orc.st_normal(A0, B0, A0 + dt * V, B0 + dt * V, 0.7, 0.2, dt)
    nx = np.array([e[1], -e[0]])
    assert np.allclose(n[:2], dt * nx, atol=1e-15)
    assert abs(n[2] + dt * (V @ nx)) < 1e-15  # n~_t = -|n~_x| V.n


@pytest.mark.parametrize("order", [2, 3, 4])
def test_vertex_velocity_weights_integrate_in_time(orc, wl, order):
    mesh, _ = wl.vortex_2d(4)
    o = orc.Oracle(mesh, order)
    W = o.ale_vertex_weights()
    X = o.st_nodes()
    verts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    M = order - 1
    for (a, b, c) in [(1.0, 0.0, 0.0), (0.3, 1.7, -0.4), (0.0, 0.0, 1.0)]:
        f = a + b * X[:, 3] ** M + c * X[:, 0] * X[:, 3] ** (M - 1)  # degree M in (xi, tau)
        for v in range(3):
            exact = a + b / (M + 1) + c * verts[v, 0] / M
            assert abs(W[v] @ f - exact) < 1e-13


@pytest.mark.parametrize("order", [2, 3])
def test_lagrangian_predictor_of_affine_density_is_steady(orc, wl, order):
    mesh, _ = wl.vortex_2d(6)
    g = np.array([0.3, -0.2])
    u = np.array([0.8, 0.5])

    def f(x):
        rho = 2.0 + x @ g
        return wl.euler_conserved(rho, np.tile(u[:, None], (1, len(rho))), np.ones_like(rho), 1.4)

    # the affine field is not periodic: use interior cells of an open mesh
    m = wl.tri_mesh(6, periodic=False, jitter=0.2, seed=3)
    Q = wl.cell_averages(m, f, n=4)
    o = orc.Oracle(m, order, params=orc.default_params(2, EULER, order=order, linear_weights=True))
    geo = o.mesh.geometry()
    cell = int(np.argmin(np.sum((geo["bary"][:, :2] - 0.5) ** 2, axis=1)))
    q, V = o.ale_predictor(Q, 0.02, cell, mode=1)
    L0 = o.Mc
    # q_hat at every tau > 0 node equals the tau = 0 value at its spatial point
    nodes = o.st_nodes()
    w0 = q[:L0]
    for k in range(L0, o.L):
        j = int(np.argmin(np.sum((nodes[:L0, :2] - nodes[k, :2]) ** 2, axis=1)))
        assert np.allclose(nodes[j, :2], nodes[k, :2])
        assert np.abs(q[k] - w0[j]).max() < 1e-12
    assert np.abs(V - u).max() < 1e-13


def test_ale_conservation_on_a_deforming_periodic_mesh(orc, wl):
    mesh, Q = wl.vortex_2d(8)
    o = orc.Oracle(mesh, 3)
    vol0 = o.mesh.geometry()["vol"]
    tot0 = vol0 @ Q
    for _ in range(3):
        Q, xyz = o.ale_step(Q, o.stable_dt(Q), mode=1)
    vol1 = o.mesh.geometry()["vol"]
    assert np.abs(xyz - mesh.xyz).max() > 1e-3                     # the mesh moved ...
    assert np.std(vol1 / vol0) > 1e-5                              # ... and deformed
    assert abs(vol1.sum() - vol0.sum()) < 1e-13                    # a periodic domain keeps its area
    assert np.abs(vol1 @ Q - tot0).max() / np.abs(tot0).max() < 1e-13


def test_ale_vortex_accuracy_on_a_deforming_mesh(orc, wl):
    """Lagrangian motion of the isentropic vortex (the moving-mesh test of
    Sec. 3.1): the deforming-mesh error at t = 0.02 is no larger than the
    fixed-mesh error of the same scheme (third order, 16x16x2 cells)."""
    import dataclasses
    mesh, Q0 = wl.vortex_2d(16)
    tf = 0.02
    errs = []
    for ale in (False, True):
        o = orc.Oracle(mesh, 3)
        Q, t = Q0.copy(), 0.0
        while t < tf - 1e-14:
            dt = min(o.stable_dt(Q), tf - t)
            Q = o.ale_step(Q, dt, mode=1)[0] if ale else o.step(Q, dt)
            t += dt
        m2 = dataclasses.replace(mesh, xyz=o.mesh.xyz())
        ex = wl.cell_averages(m2, lambda x: wl.vortex(x, t=tf), n=8)
        vol = o.mesh.geometry()["vol"]
        errs.append(vol @ np.abs(Q[:, 0] - ex[:, 0]))
    assert errs[1] < 1.2 * errs[0], errs


def test_ale_convergence_is_the_comoving_eulerian_convergence(orc, wl):
    """p10 for moving meshes: over a whole run (third order, linear weights,
    12 -> 24 cells per direction, t = 0.04) the Lagrangian errors of the
    translating density wave equal those of the Eulerian scheme on the
    co-moving stationary wave (Galilean invariance of every ALE ingredient),
    and converge at the design order.  A contact at rest relative to the mesh
    keeps the Rusanov dissipation c [q]: the fourth-order rate of both runs is
    3.24 at 16 -> 32 (measured), so the design-order bar is checked at third
    order."""
    import dataclasses
    tf = 0.04
    errs = []
    for n in (12, 24):
        mesh, _ = wl.density_wave_2d(n)
        Qm = wl.cell_averages(mesh, lambda x: _wave(wl, x, 1.0), n=6)
        Qs = wl.cell_averages(mesh, lambda x: _wave(wl, x, 0.0), n=6)
        prm = orc.default_params(2, EULER, order=3, linear_weights=True)
        a = orc.Oracle(mesh, 3, params=prm)
        nst = int(math.ceil(tf / a.stable_dt(Qm)))
        Qa, _ = a.ale_run(Qm, nst, dt=tf / nst, mode=1)
        Qb, _ = orc.Oracle(mesh, 3, params=prm).run(Qs, nst, dt=tf / nst)
        m2 = dataclasses.replace(mesh, xyz=a.mesh.xyz())
        ex = wl.cell_averages(m2, lambda x: _wave(wl, x - tf, 1.0), n=6)
        vol = a.mesh.geometry()["vol"]
        ea = vol @ np.abs(Qa[:, 0] - ex[:, 0])
        eb = vol @ np.abs(Qb[:, 0] - Qs[:, 0])
        assert abs(ea - eb) < 1e-9 * eb
        errs.append(ea)
    assert math.log2(errs[0] / errs[1]) > 2.7, errs
