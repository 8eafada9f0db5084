"""Host-side pieces of bench.py that need no GPU: the algorithmic byte and
flop model behind the roofline numbers, and the all-cores oracle timing
(worker processes stepping shares of the cells)."""
import math

import pytest


def test_algorithmic_model_counts():
    import bench
    a = bench.algorithmic(2, 4, 0, fp32=True)
    # 2D P3 Euler: n_e - 1 = 19 stencil ids, (M-1)(n_e-1) = 171 R entries
    # (Mc = 10, so 9 x 19), q_hat L nu = 20 x 4 values
    b, f = a["rec"]
    assert b == 4 * 19 + 4 * 9 * 19 + 4 * 3 * 2 + 4 * 3 * 4 + 1 + 4 * 4 + 8 * 4 + 4 * 20 * 4
    assert f > 0 and a["flux"][0] > 0 and a["update"][0] > 0
    # the matvec R dQ alone is 2 (Mc - 1)(n_e - 1) nu flops; the Picard loop
    # counts 2 nu per nonzero of P_e (116 in the unknown-node columns at 2D P3)
    assert f > 2 * 9 * 19 * 4 + 4 * 2 * 116 * 4
    # recounted without the structural zeros of P_e: below the dense count
    assert f < 2 * 9 * 19 * 4 + 4 * (2 * 10 * 20 * 4 * 2) + 20000
    # FP64 doubles the floating-point terms
    assert bench.algorithmic(2, 4, 0, fp32=False)["rec"][0] > b


def test_oracle_parallel_run_uses_worker_processes():
    import bench
    v, cores, cells, sec = bench.oracle_parallel_run("vortex2d_p2", 10, steps=1, warmup=1, nproc=2)
    assert cores == 2 and cells == 200 and v > 0 and math.isfinite(v) and sec > 0


def test_moving_mesh_oracle_baseline_line():
    """The oracle's ALE step timed beside the moving-mesh bench line: a
    bounded sample, one host thread, the baseline keys of the contract."""
    import bench
    for dim, n, shape in ((2, 6, "72 cells (6x6x2 triangles"), (3, 3, "162 cells (3^3x6 tetrahedra")):
        r = bench.ale_oracle_rate(dim=dim, n=n, steps=1)
        assert r["kind"] == "oracle" and r["cores"] == 1 and r["unit"] == "cell-updates/s"
        assert r["value"] > 0 and math.isfinite(r["value"]) and shape in r["sample"], r["sample"]


@pytest.mark.parametrize("d,M", [(2, 2), (2, 3), (3, 2)])
def test_predictor_nonzero_counts_match_exact_generator(d, M):
    """The flop model counts only the nonzeros of P_e; its counts (parsed from
    the generated header) equal a direct evaluation of the entries in exact
    rational arithmetic."""
    import importlib.util
    import os
    import bench
    spec = importlib.util.spec_from_file_location(
        "gen_pred_pattern", os.path.join(bench.ROOT, "paper_1612_09335_gb300", "csrc", "gen_pred_pattern.py"))
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    nodes = g.st_nodes(d, M)
    L0 = math.comb(M + d, d)
    nz0 = nz1 = 0
    for e in range(d):
        for k in range(len(nodes) - L0):
            for l in range(len(nodes)):
                if g.entry(d, M, nodes[L0 + k], nodes[l], e) != 0:
                    if l < L0:
                        nz0 += 1
                    else:
                        nz1 += 1
    assert bench.pred_nonzeros(d, M) == (nz0, nz1)


def test_roofline_picks_the_binding_roof():
    """A kernel whose intensity is below the ridge (peak flops / peak bytes)
    is reported against HBM, above it against the ALU peak; fractions are
    achieved / peak with achieved = algorithmic units / measured time."""
    import bench
    pk = {"hbm_gbs": 1000.0, "hbm_src": "t", "fp32_tflops": 10.0, "fp64_tflops": 1.0, "alu_src": "t"}
    alg = {"rec": (100.0, 500.0), "flux": (100.0, 5000.0), "update": (100.0, 10.0)}
    kern, dom = bench.kernel_rooflines({"k_rec_pred": 1.0, "k_flux": 2.0, "k_update": 0.5},
                                       {"rec": 1e6, "flux": 1e6, "update": 1e6}, alg, pk, fp32=True)
    assert dom == "k_flux"
    assert kern["k_rec_pred"]["bound"] == "hbm"        # 5 flop/B < ridge 10
    assert kern["k_flux"]["bound"] == "alu"            # 50 flop/B > 10
    line = bench.roofline_line(kern, dom, pk, True, None)
    assert line["bound"] == "alu" and line["unit"] == "TFLOP/s"
    assert abs(line["achieved"] - 5000.0 * 1e6 / 2e-3 / 1e12) < 1e-9
    assert abs(line["frac"] - line["achieved"] / 10.0) < 1e-12
    rec = bench.roofline_line(kern, "k_rec_pred", pk, True, None)
    assert rec["bound"] == "hbm" and abs(rec["achieved"] - 100.0 * 1e6 / 1e-3 / 1e9) < 1e-9
    # FP64: the same intensities against the FP64 ridge (1 flop/B) are ALU-bound
    k64, _ = bench.kernel_rooflines({"k_rec_pred": 1.0}, {"rec": 1e6}, alg, pk, fp32=False)
    assert k64["k_rec_pred"]["bound"] == "alu" and "fp64_frac" in k64["k_rec_pred"]


class _FakeSolver:
    """Host stand-in for a solver: forward Euler on dQ/dt = -Q with a CFL
    step that grows with time, so a step fixed at t = 0 would differ."""

    def __init__(self, noise=0.0):
        self.noise, self.t, self.Q, self.dts = noise, 0.0, None, []

    def set_state(self, Q):
        self.Q, self.t = Q.copy(), 0.0

    def step(self, dt):
        if dt == 0.0:
            dt = 1e-3 * (1.0 + self.t)
        self.dts.append(dt)
        self.Q = self.Q - dt * self.Q * (1.0 + self.noise)
        self.t += dt

    def time(self):
        return self.t

    def sync(self):
        pass

    def get_state(self):
        return self.Q.copy()


def test_accuracy_pair_follows_the_fp64_cfl_steps():
    import numpy as np

    import bench
    from paper_1612_09335_gb300 import workloads as wl
    mesh = wl.tri_mesh(4, jitter=0.1, seed=3)
    Q0 = np.tile(np.array([1.0, 0.1, -0.2, 2.5]), (mesh.nc, 1))
    a, b = _FakeSolver(noise=1e-7), _FakeSolver()
    out = bench.accuracy_pair({"fp32_mixed": a, "fp64": b}, mesh, Q0, nsteps=5)
    assert a.dts == pytest.approx(b.dts, rel=1e-12) and len(b.dts) == 5 and b.dts[-1] > b.dts[0]
    assert out["steps"] == 5 and out["dt_mean"] == pytest.approx(np.mean(b.dts))
    assert max(out["Linf_rel"]) < 1e-8 and max(out["L1_rel"]) < 1e-8
    assert len(out["conservation_drift_rel"]) == 4
