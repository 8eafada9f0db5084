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
    r = bench.ale_oracle_rate(n=6, steps=1)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["unit"] == "cell-updates/s"
    assert r["value"] > 0 and math.isfinite(r["value"]) and "72 triangles" in r["sample"]
