"""Pins of the oracle's direct ALE step on tetrahedra (Secs. 2.2-2.4 in three
space dimensions) against facts fixed by the mathematics rather than by the
oracle itself:

* the space-time normal of Eq. (detChi) for a moving triangle closes every
  moving tetrahedron: the lateral integrals of n~ equal
  (0, 0, 0, |T^n| - |T^{n+1}|), volumes by the determinant formula; a still
  face has n~ = dt ((B - A) x (C - A), 0) and a translating one
  n~_t = -|n~_x| V.n;
* V = 0 turns the ALE machinery into the Eulerian scheme (pinned separately);
* Galilean invariance: the Lagrangian step of a density wave translating
  with u = (1, 1, 1) gives the densities of the Eulerian step of the
  co-moving stationary wave on the same mesh;
* constant states stay constant under the mesh motion (GCL of Eq. gcl) and
  the mesh translates with the flow;
* the vertex-velocity weights of Eq. (NodesVel) integrate polynomials in
  tau exactly at the four reference vertices;
* the moving-element predictor of an affine density with constant velocity
  and pressure is constant in tau in the co-moving frame;
* conservation and constant total volume on a deforming periodic mesh.
"""
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


def _tet_volume(P):
    return np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]])) / 6.0


def _wave3(wl, x, u):
    s = x[:, 0] + x[:, 1] + x[:, 2]
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * s)
    return wl.euler_conserved(rho, np.full((3, len(rho)), u), np.ones_like(rho), 1.4)


def test_space_time_normals_close_a_moving_tetrahedron(orc):
    rng = np.random.default_rng(11)
    gx, gw = orc.gauss_rule(0, 2)  # tau and chi1: n~ is quadratic in tau, linear in chi
    jx, jw = orc.gauss_rule(1, 2)  # chi2: Gauss-Jacobi, weight (1 - r)
    for _ in range(20):
        P0 = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.1, 0.9, 0.1], [0.2, 0.1, 1.1]])
        P0 = P0 + 0.08 * rng.standard_normal((4, 3))
        P1 = P0 + 0.15 * rng.standard_normal((4, 3))
        dt = rng.uniform(0.01, 0.5)
        c0 = P0.mean(axis=0)
        tot = np.zeros(4)
        for k in range(4):
            A, B, C = [q for q in range(4) if q != k]
            n00 = orc.st_normal3(P0[A], P0[B], P0[C], P1[A], P1[B], P1[C], 0.0, 0.0, 0.0, dt)
            sgn = 1.0 if n00[:3] @ (P0[A] - c0) > 0 else -1.0
            for a in range(2):
                for b in range(2):
                    c1, c2 = gx[a] * (1.0 - jx[b]), jx[b]
                    for t in range(2):
                        n = orc.st_normal3(P0[A], P0[B], P0[C], P1[A], P1[B], P1[C], c1, c2, gx[t], dt)
                        tot += sgn * 0.5 * gw[a] * jw[b] * gw[t] * n
        assert np.abs(tot[:3]).max() < 1e-13
        assert abs(tot[3] - (abs(_tet_volume(P0)) - abs(_tet_volume(P1)))) < 1e-13


def test_space_time_normal3_still_and_translating_face(orc):
    A, B, C = np.array([0.2, 0.1, 0.0]), np.array([0.7, 0.5, 0.1]), np.array([0.1, 0.6, 0.4])
    cr = np.cross(B - A, C - A)
    n = orc.st_normal3(A, B, C, A, B, C, 0.3, 0.2, 0.6, 0.25)
    assert np.allclose(n, [0.25 * cr[0], 0.25 * cr[1], 0.25 * cr[2], 0.0], atol=1e-16)
    V = np.array([0.4, -1.1, 0.7])
    dt = 0.3
    n = orc.st_normal3(A, B, C, A + dt * V, B + dt * V, C + dt * V, 0.1, 0.5, 0.2, dt)
    assert np.allclose(n[:3], dt * cr, atol=1e-15)
    assert abs(n[3] + dt * (V @ cr)) < 1e-15  # n~_t = -|n~_x| V.n


@pytest.mark.parametrize("order", [2, 3, 4])
def test_ale3d_still_mesh_is_the_eulerian_step(orc, wl, order):
    mesh, Q = wl.density_wave_3d(5)
    dt = orc.Oracle(mesh, order).stable_dt(Q)
    a = orc.Oracle(mesh, order).step(Q, dt)
    b, xyz = orc.Oracle(mesh, order).ale_step(Q, dt, mode=2)
    assert np.array_equal(xyz, mesh.xyz)
    assert np.abs(a - b).max() / np.abs(a).max() < 1e-12


@pytest.mark.parametrize("order", [2, 3])
def test_ale3d_galilean_invariance(orc, wl, order):
    mesh = wl.tet_mesh(5, jitter=0.15, seed=21)
    Qm = wl.cell_averages(mesh, lambda x: _wave3(wl, x, 1.0), n=4)
    Qs = wl.cell_averages(mesh, lambda x: _wave3(wl, x, 0.0), n=4)
    prm = orc.default_params(3, EULER, order=order, linear_weights=True)
    dt = 0.004
    a, xyz = orc.Oracle(mesh, order, params=prm).ale_step(Qm, dt, mode=1)
    b = orc.Oracle(mesh, order, params=prm).step(Qs, dt)
    assert np.abs(xyz - mesh.xyz - dt).max() < 1e-15
    assert np.abs(a[:, 0] - b[:, 0]).max() < 1e-12
    assert np.abs((a[:, 1] - a[:, 0]) - b[:, 1]).max() < 1e-12
    assert np.abs(a[:, 0] - Qm[:, 0]).max() > 1e-4  # the step did change the densities


@pytest.mark.parametrize("order", [2, 3, 4])
def test_ale3d_constant_state_and_translation(orc, wl, order):
    mesh = wl.tet_mesh(4, jitter=0.15, seed=22)
    q = np.array([1.3, 0.39, -0.26, 0.13, 3.1])
    Q = np.tile(q, (mesh.nc, 1))
    o = orc.Oracle(mesh, order)
    x0 = mesh.xyz.copy()
    for _ in range(2):
        Q, xyz = o.ale_step(Q, 0.01, mode=1)
    # order 4: the Galerkin solve of Eq. (CGfinal) rounds the nodal states at ~1e-13
    assert np.abs(Q - q).max() < (1e-13 if order < 4 else 5e-13)
    assert np.abs(xyz - x0 - 0.02 * q[1:4] / q[0]).max() < 1e-14


@pytest.mark.parametrize("order", [2, 3, 4])
def test_vertex_velocity_weights_integrate_in_time_3d(orc, wl, order):
    o = orc.Oracle(wl.tet_mesh(3), order)
    W = o.ale_vertex_weights()
    X = o.st_nodes()
    verts = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    M = order - 1
    for (a, b, c, e) in [(1.0, 0.0, 0.0, 0.0), (0.3, 1.7, -0.4, 0.8), (0.0, 0.0, 0.0, 1.0)]:
        # degree M in (xi, tau)
        f = a + b * X[:, 3] ** M + c * X[:, 1] * X[:, 3] ** (M - 1) + e * X[:, 2] ** M
        for v in range(4):
            exact = a + b / (M + 1) + c * verts[v, 1] / M + e * verts[v, 2] ** M
            assert abs(W[v] @ f - exact) < 1e-13


@pytest.mark.parametrize("order", [2, 3])
def test_lagrangian_predictor_of_affine_density_is_steady_3d(orc, wl, order):
    g = np.array([0.3, -0.2, 0.25])
    u = np.array([0.8, 0.5, -0.3])

    def f(x):
        rho = 2.0 + x @ g
        return wl.euler_conserved(rho, np.tile(u[:, None], (1, len(rho))), np.ones_like(rho), 1.4)

    m = wl.tet_mesh(5, periodic=False, jitter=0.15, seed=23)
    Q = wl.cell_averages(m, f, n=4)
    o = orc.Oracle(m, order, params=orc.default_params(3, EULER, order=order, linear_weights=True))
    geo = o.mesh.geometry()
    cell = int(np.argmin(np.sum((geo["bary"] - 0.5) ** 2, axis=1)))
    q, V = o.ale_predictor(Q, 0.02, cell, mode=1)
    L0 = o.Mc
    nodes = o.st_nodes()
    w0 = q[:L0]
    for k in range(L0, o.L):
        j = int(np.argmin(np.sum((nodes[:L0, :3] - nodes[k, :3]) ** 2, axis=1)))
        assert np.allclose(nodes[j, :3], nodes[k, :3])
        assert np.abs(q[k] - w0[j]).max() < 1e-12
    assert np.abs(V - u).max() < 1e-13


def test_ale3d_conservation_on_a_deforming_periodic_mesh(orc, wl):
    mesh = wl.tet_mesh(5, jitter=0.15, seed=24)

    def f(x):
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * x[:, 0])
        vel = 0.3 * np.stack([np.sin(2 * np.pi * x[:, 1]), np.sin(2 * np.pi * x[:, 2]), np.sin(2 * np.pi * x[:, 0])])
        return wl.euler_conserved(rho, vel, np.ones_like(rho), 1.4)

    Q = wl.cell_averages(mesh, f, n=4)
    o = orc.Oracle(mesh, 3)
    vol0 = o.mesh.geometry()["vol"]
    tot0 = vol0 @ Q
    for _ in range(3):
        Q, xyz = o.ale_step(Q, o.stable_dt(Q), mode=1)
    vol1 = o.mesh.geometry()["vol"]
    assert np.abs(xyz - mesh.xyz).max() > 1e-3                     # the mesh moved ...
    assert np.std(vol1 / vol0) > 1e-5                              # ... and deformed
    assert abs(vol1.sum() - vol0.sum()) < 1e-13                    # a periodic domain keeps its volume
    assert np.abs(vol1 @ Q - tot0).max() / np.abs(tot0).max() < 1e-13


def test_lagrangian_predictor_fallback_on_the_relaxed_range(orc, wl):
    """The positivity safeguard's predictor fallback on moving meshes: a cell
    cut by the explosion's sphere whose Lagrangian Picard iteration ends on
    admissible values outside [1/2 min, 2 max] of its tau = 0 nodes' density
    or pressure (checked with the safeguard off) is sent to its cell average
    at every node (safeguard on)."""
    mesh = wl.tet_mesh(6, lo=(-1, -1, -1), hi=(1, 1, 1), periodic=False, jitter=0.15, seed=1234)
    Q0 = wl.explosion_averages(mesh, sub=4)
    cell = 343
    raw = orc.Oracle(mesh, 3, params=orc.default_params(3, EULER, order=3, positivity=False))
    dt = raw.stable_dt(Q0)
    q, _ = raw.ale_predictor(Q0, dt, cell, mode=1)
    L0 = raw.Mc
    p = 0.4 * (q[:, 4] - 0.5 * (q[:, 1] ** 2 + q[:, 2] ** 2 + q[:, 3] ** 2) / q[:, 0])
    assert (q[L0:, 0] > 0).all() and (p[L0:] > 0).all()            # admissible ...
    out = ((q[L0:, 0] < 0.5 * q[:L0, 0].min()) | (q[L0:, 0] > 2 * q[:L0, 0].max()) |
           (p[L0:] < 0.5 * p[:L0].min()) | (p[L0:] > 2 * p[:L0].max()))
    assert out.any()                                                # ... but out of range
    qs, _ = orc.Oracle(mesh, 3).ale_predictor(Q0, dt, cell, mode=1)
    assert np.array_equal(qs, np.tile(Q0[cell], (len(qs), 1)))
