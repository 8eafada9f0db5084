"""Seeded synthetic inputs: jittered simplex meshes and initial cell averages.

This module only *produces inputs* (vertex coordinates, connectivity, periodic
lengths and cell averages of initial data).  It contains none of the
reconstruction / predictor / flux arithmetic of the scheme, so both the CUDA
path and the FP64 oracle may be fed from it.

Meshes (the paper's own meshes are not available, these stand in for them):

* 2D: an n x n grid of squares, every square split along the same diagonal
  into two counter-clockwise triangles.
* 3D: an n x n x n grid of cubes, every cube split into the six Kuhn
  (Freudenthal) tetrahedra that share the main diagonal, all positively
  oriented.

Jitter: every interior vertex coordinate is moved by ``(2u-1) * a * h`` with
``u`` uniform in [0,1) drawn from SplitMix64 keyed by (seed, vertex id,
coordinate).  Vertices on the periodic seam or on the outer boundary stay
fixed.  A mesh with a non-positive cell volume is rejected.

Initial data follow the paper's test problems (Section 4): the isentropic
vortex (Eq. ShuVortIC/ShuVortDelta, rescaled to the unit square), the
explosion problem (Table RP-IC, Section 4.2.2), a smooth density wave and
the Orszag-Tang vortex (Eq. Orszag-IC).  Cell averages (Eq. cellaverage) are
taken with a collapsed Gauss rule of high degree for smooth data and with
uniform sub-simplex sampling for discontinuous data.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied element-wise to uint64 keys."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, ids: np.ndarray, coord: int, ncoord: int = 3) -> np.ndarray:
    """Uniform [0,1) numbers keyed by (seed, id, coord); counter based."""
    key = (np.uint64(seed & 0xFFFFFF) << np.uint64(40)) + ids.astype(np.uint64) * np.uint64(ncoord) \
        + np.uint64(coord)
    return (_splitmix64(key) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Mesh:
    """Plain mesh description as accepted by ``cweno_mesh_create``."""
    dim: int
    xyz: np.ndarray          # (nv, dim) float64
    cells: np.ndarray        # (nc, dim+1) int32, positively oriented
    period: np.ndarray | None  # (dim,) or None for a bounded (transmissive) box
    h: float                 # grid spacing
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nc(self) -> int:
        return int(self.cells.shape[0])

    @property
    def nv(self) -> int:
        return int(self.xyz.shape[0])

    def cell_vertices(self) -> np.ndarray:
        """Per-cell vertex coordinates (nc, dim+1, dim), periodic images unwrapped
        to the image nearest the cell's first vertex."""
        X = self.xyz[self.cells]
        if self.period is not None:
            P = np.asarray(self.period, dtype=np.float64)
            d = X - X[:, :1, :]
            X = X - P * np.round(d / P)
        return X


def _signed_volumes(X: np.ndarray) -> np.ndarray:
    dim = X.shape[2]
    E = X[:, 1:, :] - X[:, :1, :]
    det = np.linalg.det(E)
    return det / math.factorial(dim)


def tri_mesh(n: int, lo=(0.0, 0.0), hi=(1.0, 1.0), periodic: bool = True,
             jitter: float = 0.2, seed: int = 1234) -> Mesh:
    """n x n squares split into 2n^2 counter-clockwise triangles."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    L = hi - lo
    h = float(L[0] / n)
    m = n if periodic else n + 1
    I, J = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    I = I.ravel()
    J = J.ravel()
    vid = I * m + J
    xyz = np.stack([lo[0] + I * (L[0] / n), lo[1] + J * (L[1] / n)], axis=1)
    if jitter > 0:
        if periodic:
            movable = (I > 0) & (J > 0)
        else:
            movable = (I > 0) & (J > 0) & (I < n) & (J < n)
        for c in range(2):
            u = uniform01(seed, vid, c)
            off = (2.0 * u - 1.0) * jitter * (L[c] / n)
            xyz[:, c] += np.where(movable, off, 0.0)

    def v(i, j):
        if periodic:
            return (i % n) * m + (j % n)
        return i * m + j

    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ci = ci.ravel()
    cj = cj.ravel()
    v00, v10, v01, v11 = v(ci, cj), v(ci + 1, cj), v(ci, cj + 1), v(ci + 1, cj + 1)
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    cells = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    mesh = Mesh(2, xyz, cells, L.copy() if periodic else None, h,
                name=f"tri{n}{'p' if periodic else 'b'}")
    vol = _signed_volumes(mesh.cell_vertices())
    if not np.all(vol > 0):
        raise ValueError("jittered triangle mesh has a non-positive cell volume")
    return mesh


# The six Kuhn tetrahedra of the unit cube: the monotone lattice paths from
# (0,0,0) to (1,1,1), one per permutation of the axes.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def tet_mesh(n: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), periodic: bool = True,
             jitter: float = 0.15, seed: int = 1234) -> Mesh:
    """n^3 cubes, each split into 6 Kuhn tetrahedra (6 n^3 cells)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    L = hi - lo
    h = float(L[0] / n)
    m = n if periodic else n + 1
    I, J, K = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    vid = (I * m + J) * m + K
    xyz = np.stack([lo[0] + I * (L[0] / n), lo[1] + J * (L[1] / n), lo[2] + K * (L[2] / n)], axis=1)
    if jitter > 0:
        if periodic:
            movable = (I > 0) & (J > 0) & (K > 0)
        else:
            movable = (I > 0) & (J > 0) & (K > 0) & (I < n) & (J < n) & (K < n)
        for c in range(3):
            u = uniform01(seed, vid, c)
            off = (2.0 * u - 1.0) * jitter * (L[c] / n)
            xyz[:, c] += np.where(movable, off, 0.0)

    def v(i, j, k):
        if periodic:
            return ((i % n) * m + (j % n)) * m + (k % n)
        return (i * m + j) * m + k

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    tets = []
    for p in _PERMS:
        a = np.zeros(3, dtype=np.int64)
        path = [v(ci, cj, ck)]
        for ax in p:
            a[ax] += 1
            path.append(v(ci + a[0], cj + a[1], ck + a[2]))
        t = np.stack(path, axis=1)
        # odd permutations give negatively oriented tets: swap two vertices
        parity = sum(1 for x in range(3) for y in range(x + 1, 3) if p[x] > p[y]) % 2
        if parity == 1:
            t = t[:, [0, 2, 1, 3]]
        tets.append(t)
    cells = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    mesh = Mesh(3, xyz, cells, L.copy() if periodic else None, h,
                name=f"tet{n}{'p' if periodic else 'b'}")
    vol = _signed_volumes(mesh.cell_vertices())
    if not np.all(vol > 0):
        raise ValueError("jittered tetrahedral mesh has a non-positive cell volume")
    return mesh


# ----------------------------------------------------------------------------
# Quadrature used only to form initial cell averages (library routines).
# ----------------------------------------------------------------------------
def simplex_rule(dim: int, n: int):
    """Collapsed (conical product) Gauss rule on the unit simplex, n points per
    direction, exact to degree 2n-1.  Returns (points (q,dim), weights (q,))
    with weights summing to 1 (i.e. an averaging rule)."""
    from scipy.special import roots_jacobi
    xg, wg = np.polynomial.legendre.leggauss(n)
    s, ws = (xg + 1) / 2, wg / 2
    if dim == 2:
        xj, wj = roots_jacobi(n, 1.0, 0.0)
        t, wt = (xj + 1) / 2, wj / 4  # int_0^1 (1-t) f dt
        S, T = np.meshgrid(s, t, indexing="ij")
        W = np.outer(ws, wt)
        pts = np.stack([S * (1 - T), T], axis=-1).reshape(-1, 2)
        w = W.ravel()
    else:
        xj1, wj1 = roots_jacobi(n, 1.0, 0.0)
        xj2, wj2 = roots_jacobi(n, 2.0, 0.0)
        t, wt = (xj1 + 1) / 2, wj1 / 4        # weight (1-t)
        z, wz = (xj2 + 1) / 2, wj2 / 8        # weight (1-z)^2
        S, T, Z = np.meshgrid(s, t, z, indexing="ij")
        W = ws[:, None, None] * wt[None, :, None] * wz[None, None, :]
        pts = np.stack([S * (1 - T) * (1 - Z), T * (1 - Z), Z], axis=-1).reshape(-1, 3)
        w = W.ravel()
    return pts, w / w.sum()


def subsimplex_sample(dim: int, m: int):
    """Centroids of the m^dim congruent sub-triangles (2D) or a uniform
    Freudenthal sub-sampling (3D); equal weights.  For discontinuous data."""
    if dim == 2:
        pts = []
        for i in range(m):
            for j in range(m - i):
                pts.append(((i + 1 / 3) / m, (j + 1 / 3) / m))
        for i in range(m):
            for j in range(m - i - 1):
                pts.append(((i + 2 / 3) / m, (j + 2 / 3) / m))
        p = np.array(pts)
        return p, np.full(len(p), 1.0 / len(p))
    # 3D: centroids of the Kuhn sub-tets of an m-subdivided cube, kept if inside
    g = (np.arange(m) + 0.5) / m
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    P = P[P.sum(1) < 1.0]
    return P, np.full(len(P), 1.0 / len(P))


def cell_averages(mesh: Mesh, f, rule: str = "gauss", n: int = 6, chunk: int = 1 << 16,
                  only=None) -> np.ndarray:
    """Average of f(points (k,dim)) -> (k,nu) over each cell."""
    X = mesh.cell_vertices()
    if rule == "gauss":
        xi, w = simplex_rule(mesh.dim, n)
    else:
        xi, w = subsimplex_sample(mesh.dim, n)
    ids = np.arange(mesh.nc) if only is None else np.asarray(only)
    out = None
    for s in range(0, len(ids), chunk):
        c = ids[s:s + chunk]
        X0 = X[c, 0, :]
        E = X[c, 1:, :] - X0[:, None, :]          # (k, dim, dim): rows are edges
        pts = X0[:, None, :] + np.einsum("qd,kde->kqe", xi, E)
        vals = f(pts.reshape(-1, mesh.dim))
        vals = vals.reshape(len(c), len(w), -1)
        avg = np.einsum("kqv,q->kv", vals, w)
        if out is None:
            out = np.zeros((len(ids), avg.shape[1]))
        out[s:s + chunk] = avg
    return out


# ----------------------------------------------------------------------------
# Initial data (conserved variables).
# ----------------------------------------------------------------------------
def euler_conserved(rho, vel, p, gamma):
    """(rho, rho v, rho E) with rho E = p/(gamma-1) + rho |v|^2 / 2 (Eq. eos)."""
    vel = np.atleast_2d(vel)
    E = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=0)
    return np.vstack([rho[None], rho[None] * vel, E[None]]).T


def vortex(x, t=0.0, eps=5.0, centre=(0.5, 0.5), gamma=1.4, scale=10.0, L=(1.0, 1.0)):
    """Isentropic vortex of Eq. (ShuVortIC, ShuVortDelta) mapped to the unit
    square: the paper's field at x' = scale*x, translating with (1,1)."""
    xs = x[:, 0] - t
    ys = x[:, 1] - t
    # nearest periodic image of the centre
    dx = xs - centre[0]
    dy = ys - centre[1]
    dx -= L[0] * np.round(dx / L[0])
    dy -= L[1] * np.round(dy / L[1])
    r2 = (scale * dx) ** 2 + (scale * dy) ** 2
    e1 = np.exp(0.5 * (1.0 - r2))
    du = eps / (2 * np.pi) * e1 * (-scale * dy)
    dv = eps / (2 * np.pi) * e1 * (scale * dx)
    dT = -(gamma - 1.0) * eps ** 2 / (8 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    p = (1.0 + dT) ** (gamma / (gamma - 1.0))
    return euler_conserved(rho, np.vstack([1.0 + du, 1.0 + dv]), p, gamma)


def explosion(x, r0=0.5, rho_in=1.0, p_in=1.0, rho_out=0.125, p_out=0.1, gamma=1.4,
              centre=None):
    """Explosion problem (Section 4.2.2, Table RP-IC Sod states)."""
    dim = x.shape[1]
    c = np.zeros(dim) if centre is None else np.asarray(centre)
    r = np.sqrt(np.sum((x - c) ** 2, axis=1))
    inside = r < r0
    rho = np.where(inside, rho_in, rho_out)
    p = np.where(inside, p_in, p_out)
    vel = np.zeros((dim, len(r)))
    return euler_conserved(rho, vel, p, gamma)


def density_wave(x, t=0.0, amp=0.2, gamma=1.4):
    """rho = 1 + amp*sin(2 pi sum(x - t)), p = 1, v = (1,...,1): exact advection."""
    dim = x.shape[1]
    s = np.sum(x, axis=1) - dim * t
    rho = 1.0 + amp * np.sin(2 * np.pi * s)
    vel = np.ones((dim, len(rho)))
    return euler_conserved(rho, vel, np.ones_like(rho), gamma)


def linear_field(x, grad, gamma=1.4, rho0=2.0, vel=None, p0=1.0, t=0.0):
    """rho affine in x, constant velocity and pressure (advected exactly)."""
    dim = x.shape[1]
    v = np.ones(dim) * 0.5 if vel is None else np.asarray(vel)
    y = x - t * v[None, :]
    rho = rho0 + y @ np.asarray(grad)
    return euler_conserved(rho, np.repeat(v[:, None], len(rho), axis=1),
                           np.full_like(rho, p0), gamma)


def orszag_tang(x, gamma=5.0 / 3.0, bscale=math.sqrt(4 * math.pi)):
    """Orszag-Tang vortex (Eq. Orszag-IC), 9 MHD-GLM variables
    (rho, rho u, rho v, rho w, rho E, Bx, By, Bz, psi); Gaussian units,
    rho E = p/(gamma-1) + rho|v|^2/2 + |B|^2/(8 pi)."""
    X, Y = x[:, 0], x[:, 1]
    rho = np.full_like(X, gamma * gamma)
    u, v, w = -np.sin(Y), np.sin(X), np.zeros_like(X)
    p = np.full_like(X, gamma)
    Bx, By, Bz = -bscale * np.sin(Y), bscale * np.sin(2 * X), np.zeros_like(X)
    E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v + w * w) + (Bx * Bx + By * By + Bz * Bz) / (8 * np.pi)
    return np.stack([rho, rho * u, rho * v, rho * w, E, Bx, By, Bz, np.zeros_like(X)], axis=1)


def alfven_wave(x, t=0.0, gamma=5.0 / 3.0, amp=0.1):
    """Circularly polarised Alfven wave on the periodic unit square: an exact
    travelling solution of ideal MHD (Gaussian units) with wave vector
    2 pi (1, 1), background rho = 1, p = 0.1 and |B0| = sqrt(4 pi) along the
    diagonal (Alfven speed 1)."""
    ca = sa = math.sqrt(0.5)
    rho0, p0, B0 = 1.0, 0.1, math.sqrt(4 * math.pi)
    va = B0 / math.sqrt(4 * math.pi * rho0)
    kmag = 2 * np.pi * math.sqrt(2.0)
    phase = 2 * np.pi * (x[:, 0] + x[:, 1]) - kmag * va * t
    b_perp = amp * B0 * np.sin(phase)
    b_z = amp * B0 * np.cos(phase)
    v_perp = -b_perp / math.sqrt(4 * math.pi * rho0)
    v_z = -b_z / math.sqrt(4 * math.pi * rho0)
    Bx = B0 * ca - b_perp * sa
    By = B0 * sa + b_perp * ca
    u = -v_perp * sa
    v = v_perp * ca
    rho = np.full_like(phase, rho0)
    p = np.full_like(phase, p0)
    E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v + v_z * v_z) + (Bx * Bx + By * By + b_z * b_z) / (8 * np.pi)
    return np.stack([rho, rho * u, rho * v, rho * v_z, E, Bx, By, b_z, np.zeros_like(phase)], axis=1)


# ----------------------------------------------------------------------------
# Named workloads (synthetic stand-ins for the paper's test problems).
# ----------------------------------------------------------------------------
def vortex_2d(n=32, jitter=0.2, seed=1234, eps=5.0):
    """Periodic unit square, n x n x 2 jittered triangles, isentropic vortex."""
    mesh = tri_mesh(n, periodic=True, jitter=jitter, seed=seed)
    Q = cell_averages(mesh, lambda x: vortex(x, eps=eps), n=6)
    return mesh, Q


def explosion_2d(n=512, jitter=0.2, seed=1234):
    """[-1,1]^2 with transmissive boundaries, circular explosion (r < 0.5)."""
    mesh = tri_mesh(n, lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=False, jitter=jitter, seed=seed)
    Q = explosion_averages(mesh)
    return mesh, Q


def explosion_averages(mesh, r0=0.5, centre=None, p_in=1.0, sub=16, **kw):
    """Cell averages of the explosion data: the point value for cells that
    lie entirely on one side of the circle, uniform sub-simplex sampling for
    the cells it cuts.  The circle must not cross a periodic seam."""
    c = np.zeros(mesh.dim) if centre is None else np.asarray(centre, dtype=np.float64)

    def f(x):
        return explosion(x, r0=r0, p_in=p_in, centre=c, **kw)

    X = mesh.cell_vertices()
    r = np.sqrt(np.sum((X - c) ** 2, axis=2))
    Q = f(X.mean(axis=1))
    cut = np.where((r.min(axis=1) < r0 + mesh.h) & (r.max(axis=1) >= r0 - mesh.h))[0]
    if len(cut):
        Q[cut] = cell_averages(mesh, f, rule="sub", n=sub, only=cut)
    return Q


def density_wave_3d(n=64, jitter=0.15, seed=1234):
    mesh = tet_mesh(n, periodic=True, jitter=jitter, seed=seed)
    Q = cell_averages(mesh, lambda x: density_wave(x), n=4)
    return mesh, Q


def density_wave_2d(n=32, jitter=0.2, seed=1234):
    mesh = tri_mesh(n, periodic=True, jitter=jitter, seed=seed)
    Q = cell_averages(mesh, lambda x: density_wave(x), n=6)
    return mesh, Q


def orszag_tang_2d(n=724, jitter=0.2, seed=1234):
    L = 2 * math.pi
    mesh = tri_mesh(n, lo=(0.0, 0.0), hi=(L, L), periodic=True, jitter=jitter, seed=seed)
    Q = cell_averages(mesh, orszag_tang, n=4)
    return mesh, Q


# Configurations of the benchmarked workloads (name -> parameters).
CONFIGS = {
    "vortex2d_p2": dict(dim=2, order=3, pde="euler", n=32, steps=10, cfl=0.5),
    "explosion2d_p3": dict(dim=2, order=4, pde="euler", n=512, steps=100, cfl=0.5),
    "densitywave3d_p2": dict(dim=3, order=3, pde="euler", n=64, steps=50, cfl=1.0 / 3.0),
    "orszagtang2d_p3": dict(dim=2, order=4, pde="mhd", n=724, steps=100, cfl=0.5),
}


def make_workload(name: str, n: int | None = None):
    cfg = CONFIGS[name]
    n = cfg["n"] if n is None else n
    if name == "vortex2d_p2":
        return vortex_2d(n)
    if name == "explosion2d_p3":
        return explosion_2d(n)
    if name == "densitywave3d_p2":
        return density_wave_3d(n)
    if name == "orszagtang2d_p3":
        return orszag_tang_2d(n)
    raise KeyError(name)


def serving_stream(nreq=512, seed=42, rate=None, nmin=1000, nmax=200000):
    """Seeded request stream: (arrival time, n, order, kind, params) tuples.
    Poisson arrivals with the given rate (requests/s; None -> all at t=0),
    log-uniform cell counts (n = round(sqrt(N/2))), orders P1..P3 and either a
    vortex or an explosion initial state on a periodic unit square."""
    rng = np.random.default_rng(seed)
    # arrival times from their own stream: the requests are the same at any rate
    rng_t = np.random.default_rng([seed, 1])
    out = []
    t = 0.0
    for k in range(nreq):
        if rate:
            t += rng_t.exponential(1.0 / rate)
        N = math.exp(rng.uniform(math.log(nmin), math.log(nmax)))
        n = max(8, int(round(math.sqrt(N / 2))))
        order = int(rng.integers(2, 5))
        if rng.uniform() < 0.5:
            kind = "vortex"
            params = dict(centre=tuple(rng.uniform(0.25, 0.75, 2)), eps=float(rng.uniform(1, 5)))
        else:
            kind = "explosion"
            params = dict(r0=float(rng.uniform(0.2, 0.4)), pratio=float(rng.uniform(5, 20)))
        out.append(dict(id=k, t=t, n=n, order=order, kind=kind, params=params, seed=1234 + k))
    return out


def serving_request_inputs(req):
    """Mesh and initial cell averages of one request of `serving_stream`
    (collapsed Gauss rule with 3 x 3 points for the vortex, 4 x 4 x 2
    sub-triangle samples for the explosion: initial data of a throughput
    workload, generated for tens of millions of cells)."""
    mesh = tri_mesh(req["n"], periodic=True, jitter=0.2, seed=req["seed"])
    if req["kind"] == "vortex":
        c = req["params"]["centre"]
        Q = cell_averages(mesh, lambda x: vortex(x, eps=req["params"]["eps"], centre=c), n=3)
    else:
        pr = req["params"]["pratio"]
        Q = explosion_averages(mesh, r0=req["params"]["r0"], centre=(0.5, 0.5), p_in=0.1 * pr,
                               sub=4)
    return mesh, Q
