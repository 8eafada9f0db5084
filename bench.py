#!/usr/bin/env python
"""ADER-CWENO cell-updates/s on GB300.

One bench "step" is one full ADER-CWENO time step (reconstruction +
predictor, face fluxes, conservative update and the CFL bound for the next
step) over the whole mesh of the workload, run through the C ABI.  The
default workload is the 2D explosion: 512 x 512 x 2 = 524,288 jittered
triangles on [-1,1]^2 with transmissive boundaries, fourth order (P3), Euler,
CFL 0.5, FP32-mixed arithmetic; the FP64 mode is timed beside it.

Prints ONE JSON line.  `value` is whole-job cell-updates/s (N GPUs run
independent replicas, weak scaling); `e2e` is the same metric with the
state uploaded from and downloaded to pinned host memory every step.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "explosion2d_p3": dict(dim=2, order=4, pde=0, n=512, desc="512x512x2 jittered triangles on [-1,1]^2, "
                           "transmissive, circular explosion, Euler gamma 1.4, P3, CFL 0.5"),
    "densitywave3d_p2": dict(dim=3, order=3, pde=0, n=64, desc="64^3 x 6 jittered Kuhn tetrahedra, periodic "
                             "unit cube, density wave, Euler, P2, CFL 1/3"),
    "orszagtang2d_p3": dict(dim=2, order=4, pde=1, n=724, desc="724x724x2 jittered triangles, periodic "
                            "[0,2pi]^2, Orszag-Tang, MHD-GLM gamma 5/3 c_h 2, P3, CFL 0.5"),
    "explosion2d_p4": dict(dim=2, order=5, pde=0, n=512, desc="512x512x2 jittered triangles on [-1,1]^2, "
                           "transmissive, circular explosion, Euler gamma 1.4, P4 (fifth order), CFL 0.5"),
    "densitywave3d_p4": dict(dim=3, order=5, pde=0, n=32, desc="32^3 x 6 jittered Kuhn tetrahedra, periodic "
                             "unit cube, density wave, Euler, P4 (fifth order), CFL 1/3"),
    "vortex2d_p2": dict(dim=2, order=3, pde=0, n=32, desc="32x32x2 jittered triangles, periodic unit "
                        "square, isentropic vortex, Euler, P2, CFL 0.5"),
}
METRIC = "ADER-CWENO cell-updates/s"


def make_inputs(name, n=None):
    from paper_1612_09335_gb300 import workloads as wl
    cfg = WORKLOADS[name]
    n = cfg["n"] if n is None else n
    if name in ("explosion2d_p3", "explosion2d_p4"):
        return wl.explosion_2d(n)
    if name in ("densitywave3d_p2", "densitywave3d_p4"):
        return wl.density_wave_3d(n)
    if name == "orszagtang2d_p3":
        return wl.orszag_tang_2d(n)
    return wl.vortex_2d(n)


# ------------------------------------------------------------ algorithmic counts
def mcal(M, d):
    return math.comb(M + d, d)


def pred_nonzeros(d, M):
    """(nonzeros of P_e in the tau = 0 columns, nonzeros in the unknown-node
    columns), summed over the d directions, from the exact zero pattern of the
    closed-form predictor matrices (csrc/pred_pattern.h, generated in exact
    rational arithmetic).  Zeros of P_e are structural, not the method's work."""
    import re
    txt = open(os.path.join(ROOT, "paper_1612_09335_gb300", "csrc", "pred_pattern.h")).read()
    m = re.search(r"struct PredPattern<%d, %d> \{.*?return \((.*?)\)\[" % (d, M), txt, re.S)
    bits = "".join(re.findall(r'"([01]+)"', m.group(1)))
    L, L0 = mcal(M, d + 1), mcal(M, d)
    L1 = L - L0
    nz0 = nz1 = 0
    for e in range(d):
        for k in range(L1):
            row = bits[(e * L1 + k) * L:(e * L1 + k + 1) * L]
            nz0 += row[:L0].count("1")
            nz1 += row[L0:].count("1")
    return nz0, nz1


def phys_flops(d, pde):
    """Flops of the pointwise physics (an FMA counts 2, a division, reciprocal
    or square root 1): primitive variables from a state, the normal flux
    along a general direction, the flux along a coordinate axis, the largest
    signal speed along a unit normal and over all directions, the pressure."""
    if pde == 0:
        return dict(prim=3 * d + 3, fluxn=5 * d + 2, axis=d + 4, smax=2 * d + 4, speed=2 * d + 4,
                    pressure=2 * d + 4)
    return dict(prim=26, fluxn=42, axis=30, smax=25, speed=20, pressure=14)


def algorithmic(dim, order, pde, fp32=True, flux=0):
    """Algorithmic bytes and flops per unit of each kernel (a unit is a cell
    for the reconstruction + predictor and the update kernels, a face for the
    flux kernel).  Bytes count each datum the method must move once (stencil
    neighbours' states are the same data as their own, read once); flops
    count the method's arithmetic, 2 per FMA, with the exact zeros of the
    predictor matrices skipped (they are structural in the closed form of the
    Galerkin predictor), the positivity safeguard included (on by default and
    timed).  `flux`: 0 quadrature Rusanov, 1 Osher-type, 2 quadrature-free."""
    d, M = dim, order - 1
    nv = 9 if pde == 1 else d + 2
    Mc, L = mcal(M, d), mcal(M, d + 1)
    ne1, MC1, NS = d * Mc - 1, Mc - 1, d + 1
    L0 = Mc
    L1 = L - L0
    r = 4 if fp32 else 8
    nqs = (M + 1) ** (d - 1)
    nqt = M + 1
    niter = M + 1
    ph = phys_flops(d, pde)
    nz0, nz1 = pred_nonzeros(d, M)
    rec_bytes = (4 * ne1 + r * MC1 * ne1 + 4 * NS * d + r * NS * d * d + 1 + r * d * d + 8 * nv + r * L * nv)
    node_flux = nv + ph["prim"] + d * (ph["fluxn"] + nv)      # q = Qbar + dev, G_e - G_e(Qbar) per direction
    rec_flops = ((ne1 + NS * d) * nv                           # stencil differences
                 + 2 * MC1 * ne1 * nv                          # P_opt = R dQ (Eq. CWENO:Popt)
                 + 2 * NS * d * d * nv                         # sectorial gradients (Eq. CWENO:Ps)
                 + nv * (2 * d * NS + MC1)                     # P_0 (Eq. CWENO:P0)
                 + nv * (2 * MC1 * MC1 + 2 * MC1 + NS * (2 * d * d + 2 * d))  # indicators (Eq. Sigma_lm)
                 + nv * (8 * (NS + 1) + 1)                     # nonlinear weights (Eq. weights2)
                 + nv * (MC1 + 2 * d * NS)                     # w = sum omega P
                 + L0 * nv * 2 * MC1                           # w at the tau = 0 nodes
                 + L0 * (ph["pressure"] + 6)                   # positivity checks at the lattice nodes
                 + ph["prim"] + d * ph["fluxn"]                # G_e(Qbar)
                 + L0 * node_flux + 2 * nz0 * nv               # fixed part: -sum_e P_e[:, tau=0] G_e
                 + L1 * nv * (2 * MC1 + 1)                     # known part (C0 E) w
                 + niter * (L1 * node_flux + 2 * nz1 * nv)     # Picard iterations (Eq. CGfinal)
                 + L1 * (nv + ph["pressure"] + 3))             # predictor admissibility
    # per face: both sides' predictors and cell averages (each cell's read
    # once over its d + 1 faces), the two cell ids and codes, the unit normal,
    # |f| n and |f| (FP64), the face integral (FP64)
    flux_bytes_face = (2 / (d + 1)) * (r * L * nv + 8 * nv) + 4 + 4 + 2 + r * d + 8 * d + 8 + 8 * nv
    npts = nqt * nqs
    point = (2 * nv + 2 * ph["prim"] + 4 + 2 * d * ph["axis"] + 3 * d * nv)  # traces + averages, both fluxes
    if flux == 1:  # Osher-type: 3-point path rule of |A_n| dq
        point += 3 * (nv + 4 * d + 45 + 4 * nv) + 3 * nv
    else:
        point += 2 * ph["smax"] + 2 + 3 * nv
    if flux == 2:  # quadrature-free: one pass over each side's L nodes
        flux_flops_face = (2 * L * (nv + ph["prim"] + d * ph["axis"] + d * nv * 3 + 2 * nv)
                           + 2 * ph["prim"] + 2 * ph["smax"] + 4 * nv + nv * (2 * d + 3))
    else:
        flux_flops_face = 2 * npts * L * nv * 2 + npts * point + nv * (2 * d + 3)
    # face ids, face integrals (each read by its two cells: once per face),
    # Q read and written (FP64), the FP32 hi/lo copies written, 1/|T| and h
    upd_bytes = 4 * (d + 1) + (d + 1) / 2 * 8 * nv + 16 * nv + (8 * nv if fp32 else 0) + 16
    upd_flops = (d + 1) * nv + 2 * nv + nv + ph["pressure"] + ph["speed"] + 4
    return dict(rec=(rec_bytes, rec_flops), flux=(flux_bytes_face, flux_flops_face), update=(upd_bytes, upd_flops))


def peaks(fma=None):
    """Roofline denominators: the measured HBM copy bandwidth
    (MEASURED_PEAKS.json, else the fallback 6800 GB/s) and the FP32 / FP64 FMA
    rates measured on this device by cweno_measure_fma_peak (`fma`), else
    derived from the SM count, 128 FP32 lanes per SM, 2 flops per FMA and the
    maximum SM clock (FP64: 1/64 of that)."""
    p = {"hbm_gbs": 6800.0, "hbm_src": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        mp = json.load(open(path))
        p = {"hbm_gbs": float(mp["hbm_gbs"]), "hbm_src": "measured (MEASURED_PEAKS.json copy bandwidth)",
             "sm_max_mhz": float(mp.get("sm_max_mhz", 2070))}
    p.setdefault("sm_max_mhz", 2070.0)
    nsm = 152
    try:
        import torch
        if torch.cuda.is_available():
            nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    except Exception:
        pass
    p["sm_count"] = nsm
    derived = nsm * 128 * 2 * p["sm_max_mhz"] * 1e6 / 1e12
    if fma:
        p["fp32_tflops"], p["fp64_tflops"] = fma["fp32_tflops"], fma["fp64_tflops"]
        p["alu_src"] = (f"measured: FMA-chain kernel on {nsm} SMs at a median {fma.get('sm_mhz')} MHz "
                        f"(derived FP32 at the max clock: {derived:.1f} TFLOP/s)")
    else:
        p["fp32_tflops"], p["fp64_tflops"] = derived, derived / 64
        p["alu_src"] = f"derived: {nsm} SM x 128 FP32 lanes x 2 x {p['sm_max_mhz']:.0f} MHz (FP64 1/64)"
    return p


def kernel_rooflines(kernel_ms, units, alg, pk, fp32=True):
    """Per kernel: algorithmic GB/s and TFLOP/s from its average launch time,
    the HBM and pipe fractions, and which roof binds by arithmetic intensity
    against the ridge of the measured peaks.  Returns (kernels, dominant)."""
    alu_peak = pk["fp32_tflops"] if fp32 else pk["fp64_tflops"]
    ridge = alu_peak * 1e12 / (pk["hbm_gbs"] * 1e9)
    out = {}
    tot = sum(kernel_ms.values())
    for name, ms in kernel_ms.items():
        key = {"k_rec_pred": "rec", "k_flux": "flux", "k_update": "update"}[name]
        b, f = alg[key]
        dur = ms / 1e3
        gbs = b * units[key] / dur / 1e9
        tf = f * units[key] / dur / 1e12
        inten = f / b
        bound = "alu" if inten > ridge else "hbm"
        out[name] = {"ms": ms, "share": ms / tot if tot else None, "bytes_per_unit": b, "flops_per_unit": f,
                     "units": units[key], "intensity_flop_per_byte": inten, "GB/s": gbs, "TFLOP/s": tf,
                     "hbm_frac": gbs / pk["hbm_gbs"], ("fp32_frac" if fp32 else "fp64_frac"): tf / alu_peak,
                     "bound": bound}
    dom = max(out, key=lambda k: out[k]["ms"])
    return out, dom


def roofline_line(kern, dom, pk, fp32, traffic):
    k = kern[dom]
    fr = "fp32_frac" if fp32 else "fp64_frac"
    if k["bound"] == "hbm":
        return {"bound": "hbm", "achieved": k["GB/s"], "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": k["hbm_frac"],
                "traffic": traffic, "kernel": dom, "peak_src": pk["hbm_src"], fr: k[fr],
                "intensity_flop_per_byte": k["intensity_flop_per_byte"]}
    return {"bound": "alu", "achieved": k["TFLOP/s"], "peak": pk["fp32_tflops"] if fp32 else pk["fp64_tflops"],
            "unit": "TFLOP/s", "frac": k[fr], "traffic": traffic, "kernel": dom,
            "peak_src": pk["alu_src"] + (" (FP32 FMA)" if fp32 else " (FP64 FMA)"), "hbm_frac": k["hbm_frac"],
            "intensity_flop_per_byte": k["intensity_flop_per_byte"]}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cuh",):
        h.update(open(os.path.join(ROOT, "paper_1612_09335_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    for r in rec.get("entries", []):
        if r.get("kernel") == kernel and r.get("workload") == workload and r.get("source") == kernel_source_hash():
            return r.get("dram_bytes_per_launch")
    return None


# ---------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0, period_ms=50):
        self.rows = []
        self.proc = None
        self.t = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", f"-lms={period_ms}"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [r for t, r in self.rows if t0 - 0.06 <= t <= t1 + 0.06] or [r for _, r in self.rows[-3:]]
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


# --------------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """The largest x over the ranks of the default process group (a timed
    region's duration: the job is as slow as its slowest replica); x itself
    without a group.  NCCL reduces a device tensor, other backends a host one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ws: int, units_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of ws replicas (weak scaling): all units processed
    by all ranks over the slowest rank's time."""
    return ws * units_per_rank * steps / seconds


def cpu_baseline_run(name, seconds_budget=20.0, cells_hint=None, cw=None):
    """Time the FP64 oracle (single host thread, as it stands) on a bounded
    sample of the workload: the same scheme on a coarser mesh of the same
    family, one untimed warm step (lazy per-cell setup), then timed steps.
    With `cw` (the binding) the CUDA path in both precisions runs the same
    steps from the same data and its per-variable errors against the
    oracle's result are returned under "vs_oracle"."""
    import oracle
    from paper_1612_09335_gb300 import workloads as wl
    cfg = WORKLOADS[name]
    per_cell = {(2, 4, 0): 200e-6, (2, 3, 0): 65e-6, (3, 3, 0): 400e-6, (2, 4, 1): 900e-6}.get(
        (cfg["dim"], cfg["order"], cfg["pde"]), 300e-6)
    target = cells_hint or max(512, int(seconds_budget / 3 / per_cell))
    if cfg["dim"] == 2:
        n = max(8, int(math.sqrt(target / 2)))
    else:
        n = max(4, int(round((target / 6) ** (1 / 3))))
    mesh, Q = make_inputs(name, n)
    Q0 = Q.copy()
    o = oracle.Oracle(mesh, cfg["order"], cfg["pde"])
    dt = o.stable_dt(Q)
    Q = o.step(Q, dt)
    steps = 0
    t0 = time.perf_counter()
    while True:
        Q = o.step(Q, dt)
        steps += 1
        if time.perf_counter() - t0 > seconds_budget * 0.5 or steps >= 3:
            break
    el = time.perf_counter() - t0
    out = dict(value=mesh.nc * steps / el, unit="cell-updates/s", cores=1, kind="oracle",
               sample=f"{mesh.nc} cells ({n}-cell grid of the same workload family), {steps} steps after one "
                      f"untimed warm step, single host thread")
    if cw is not None:
        vs = {"cells": mesh.nc, "steps": steps + 1, "dt": dt,
              "reference": "the FP64 oracle's result on this sample (same mesh, initial data and time step)"}
        m = cw.Mesh.from_workload(mesh)
        for prec, key in ((cw.FP64, "fp64"), (cw.FP32_MIXED, "fp32_mixed")):
            sv = cw.Solver(m, cfg["order"], cfg["pde"], prec)
            sv.set_state(Q0)
            for _ in range(steps + 1):
                sv.step(dt)
            acc = accuracy_metrics(mesh, Q0, sv.get_state(), Q)
            vs[key] = {"L1_rel": acc["L1_rel"], "Linf_rel": acc["Linf_rel"]}
            sv.close()
        m.close()
        out["vs_oracle"] = vs
    # the same oracle on all host cores (worker processes), a 4x larger sample
    n4 = 2 * n if cfg["dim"] == 2 else int(round(n * 4 ** (1 / 3)))
    v, cores, cells, sec = oracle_parallel_run(name, n4, steps=3)
    out["all_cores"] = dict(value=v, unit="cell-updates/s", cores=cores, kind="oracle",
                            sample=f"{cells} cells, 3 steps after one untimed warm step, {cores} worker processes "
                                   f"each stepping a contiguous share of the cells")
    return out


# The oracle on all host cores: worker processes (spawned: this process may
# already hold a CUDA context) each step a contiguous share of the cells of
# the same sample with the unmodified oracle; the parent gathers the state
# between steps.
_ORC = None


def _oracle_worker_init(name, n):
    global _ORC
    import oracle
    cfg = WORKLOADS[name]
    mesh, _ = make_inputs(name, n)
    _ORC = oracle.Oracle(mesh, cfg["order"], cfg["pde"])


def _oracle_worker_step(args):
    Q, dt, ids = args
    return _ORC.step(Q, dt, ids=ids)


def oracle_parallel_run(name, n, steps, warmup=1, nproc=None):
    """Cell-updates/s of the FP64 oracle on `nproc` processes (default: all
    host cores) for `steps` timed steps after `warmup` untimed ones (the
    first builds the per-cell setup lazily).  Returns (value, cores, cells,
    seconds)."""
    import multiprocessing
    import numpy as np
    import oracle
    oracle.build()
    cfg = WORKLOADS[name]
    nproc = nproc or os.cpu_count() or 1
    mesh, Q = make_inputs(name, n)
    o = oracle.Oracle(mesh, cfg["order"], cfg["pde"])
    chunks = np.array_split(np.arange(mesh.nc, dtype=np.int64), nproc)
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(nproc, initializer=_oracle_worker_init, initargs=(name, n)) as pool:
        def one(Q):
            dt = o.stable_dt(Q)
            return np.concatenate(pool.map(_oracle_worker_step, [(Q, dt, c) for c in chunks]))
        for _ in range(max(1, warmup)):
            Q = one(Q)
        t0 = time.perf_counter()
        for _ in range(steps):
            Q = one(Q)
        el = time.perf_counter() - t0
    return mesh.nc * steps / el, nproc, mesh.nc, el


def serving_run(cw, nreq, steps=50, seed=42, max_slots=256, seq_sample=16, loads=(0.5, 0.8)):
    """Serving mix shaped like the paper-scale serving workload: independent 2D
    Euler solves (periodic meshes of 1k-200k cells, log-uniform; orders P1-P3;
    vortex or explosion data), 50 steps at CFL 0.5, FP32-mixed.  Phase 1 runs
    them as a closed batch to measure capacity; phase 2 submits them as a
    seeded Poisson stream at each fraction `loads` of that capacity and
    reports latency percentiles (submit to completion, host wall clock, setup
    included).  The sequential baseline runs a sample one after another
    through the solver API in FP64 (setup included)."""
    import numpy as np
    from paper_1612_09335_gb300 import workloads as wl
    stream = wl.serving_stream(nreq=nreq, seed=seed, rate=None)
    inputs = [wl.serving_request_inputs(r) for r in stream]
    cells = sum(m.nc for m, _ in inputs)
    # phase 1: closed batch
    srv = cw.Server(max_slots=max_slots)
    t0 = time.perf_counter()
    ids = [srv.submit(m, Q, r["order"], 0.5, steps) for (m, Q), r in zip(inputs, stream)]
    srv.drain(3600)
    t_closed = time.perf_counter() - t0
    ok = sum(srv.poll(i)[0] == cw.REQ_DONE for i in ids)
    st1 = srv.stats()
    srv.close()
    cap = nreq / t_closed
    out = {"requests": nreq, "steps_per_request": steps, "cells_total": cells, "completed_closed": ok,
           "closed_batch_s": t_closed, "closed_cell_updates_per_s": cells * steps / t_closed,
           "capacity_req_per_s": cap, "max_slots": max_slots,
           "closed_member_steps_per_tick": st1["member_steps"] / max(1, st1["ticks"]), "open_loop": {}}
    # phase 2: Poisson arrivals at fractions of that capacity
    peak = st1["peak_running"]
    for load in loads:
        arr = wl.serving_stream(nreq=nreq, seed=seed, rate=load * cap)
        srv = cw.Server(max_slots=max_slots)
        t0 = time.perf_counter()
        ids = []
        for (m, Q), r in zip(inputs, arr):
            dt_wait = r["t"] - (time.perf_counter() - t0)
            if dt_wait > 0:
                time.sleep(dt_wait)
            ids.append(srv.submit(m, Q, r["order"], 0.5, steps))
        srv.drain(3600)
        t_open = time.perf_counter() - t0
        lat, lat_nc = [], []
        for i, (m, _) in zip(ids, inputs):
            st, _, l = srv.poll(i)
            if st == cw.REQ_DONE:
                lat.append(l)
                lat_nc.append(m.nc)
        stats = srv.stats()
        srv.close()
        peak = max(peak, stats["peak_running"])
        bands = {}
        for lo, hi, key in ((0, 16384, "below_16k_cells"), (16384, 1 << 62, "from_16k_cells")):
            sel = [l for l, n in zip(lat, lat_nc) if lo <= n < hi]
            if sel:
                bands[key] = {"requests": len(sel), "p50_latency_s": float(np.percentile(sel, 50)),
                              "p99_latency_s": float(np.percentile(sel, 99))}
        lat = np.array(lat)
        out["open_loop"][f"{load:.1f}x_capacity"] = {
            "arrival_rate_req_per_s": load * cap, "open_wall_s": t_open, "completed_open": len(lat),
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "open_cell_updates_per_s": stats["cell_updates"] / t_open, "latency_by_size": bands,
            "member_steps_per_tick": stats["member_steps"] / max(1, stats["ticks"])}
    hi = out["open_loop"][f"{loads[-1]:.1f}x_capacity"]
    out["p50_latency_s"], out["p99_latency_s"] = hi["p50_latency_s"], hi["p99_latency_s"]
    out["peak_running"] = int(peak)
    # sequential FP64 per-solve baseline on a sample of the same requests
    k = min(seq_sample, nreq)
    seq_cells = 0
    ts = time.perf_counter()
    for (m, Q), r in list(zip(inputs, stream))[:k]:
        sv = cw.Solver(cw.Mesh.from_workload(m), r["order"], cw.EULER, cw.FP64, cfl=0.5)
        sv.set_state(Q)
        sv.run(steps)
        sv.get_state()
        sv.close()
        seq_cells += m.nc
    t_seq = time.perf_counter() - ts
    out.update({"sequential_fp64_cell_updates_per_s": seq_cells * steps / t_seq, "sequential_sample_requests": k,
                "note": "wall clock includes host setup (mesh on the host; stencils, sectors and least-squares "
                        "inverses on the device); top-level p50/p99 are those of the highest load"})
    return out


def accuracy_metrics(mesh, Q0, qa, qb):
    """Per-variable L1 (volume weighted, relative to the variable's L1 norm)
    and L_inf (relative to its max) errors of qa against qb, a variable whose
    norm is below 1 % of the largest variable's measured at that 1 % (the
    rule of the FP32 parity tests: psi of MHD-GLM starts at zero), and the
    drift of sum |T_i| Q_i in qa relative to the larger of the totals and the
    L1 norms (floored at 1e-6 of the largest, so identically zero variables
    are measured at the state's scale)."""
    import numpy as np
    Xv = mesh.cell_vertices()
    vol = np.abs(np.linalg.det(Xv[:, 1:] - Xv[:, :1])) / math.factorial(mesh.dim)
    n1 = vol @ np.abs(qb)
    ninf = np.abs(qb).max(axis=0)
    l1 = (vol @ np.abs(qa - qb)) / np.maximum(np.maximum(n1, 1e-2 * n1.max()), 1e-300)
    linf = np.abs(qa - qb).max(axis=0) / np.maximum(np.maximum(ninf, 1e-2 * ninf.max()), 1e-300)
    tot0 = vol @ Q0
    scale = np.maximum(np.maximum(np.abs(tot0), vol @ np.abs(Q0)), vol @ np.abs(qa))
    scale = np.maximum(scale, 1e-6 * scale.max())
    drift = np.abs(vol @ qa - tot0) / scale
    return {"L1_rel": [float(x) for x in l1], "Linf_rel": [float(x) for x in linf],
            "conservation_drift_rel": [float(x) for x in drift]}


def accuracy_pair(solvers, mesh, Q0, nsteps=10):
    """FP32-mixed against the FP64 mode after nsteps steps: the FP64 solver
    takes its device CFL step, FP32-mixed follows with the same step sizes;
    `solvers` maps "fp32_mixed" / "fp64" to live solvers of the same fixed
    mesh and scheme (set_state restarts them)."""
    import numpy as np
    a, b = solvers["fp32_mixed"], solvers["fp64"]
    a.set_state(Q0)
    b.set_state(Q0)
    dts = []
    for _ in range(nsteps):
        t0 = b.time()
        b.step(0.0)
        dts.append(b.time() - t0)
        a.step(dts[-1])
    a.sync()
    b.sync()
    out = accuracy_metrics(mesh, Q0, a.get_state(), b.get_state())
    out.update({"reference": "FP64 mode of the same solver (itself parity-tested against the FP64 oracle to "
                             "1e-12, one step at full size on sampled cells)", "steps": nsteps,
                "dt_mean": float(np.mean(dts))})
    return out


def time_solver(s, stream, barrier, Q0, k, warm=3):
    """k steps with the device CFL bound after `warm` untimed ones, CUDA events
    on the solver's stream; returns (ms per step, per-kernel mean ms)."""
    import torch
    s.set_state(Q0)
    for _ in range(warm):
        s.step(0.0)
    s.sync()
    s.set_state(Q0)
    s.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(k):
        s.step(0.0)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    kms, kn = s.profile_read()
    s.profile(False)
    s.sync()
    names = ("k_rec_pred", "k_flux", "k_update")
    return ms / k, {names[q]: kms[q] / kn[q] for q in range(3) if kn[q]}, int(sum(kn))


def workload_rate(cw, name, stream, barrier, pk, steps=10, flux=0, precisions=None, inputs=None):
    """Cell-updates/s of a benchmark workload in both precisions (same
    timing method: CUDA events on the solver stream, device CFL step), the
    per-kernel rooflines of each, and the accuracy of the FP32-mixed mode
    against the FP64 mode; `flux` selects the face flux (0 Rusanov, 1
    Osher-type, 2 quadrature-free Rusanov)."""
    cfg = WORKLOADS[name]
    mesh, Q0 = make_inputs(name) if inputs is None else inputs
    m = cw.Mesh.from_workload(mesh)
    res = {"cells": mesh.nc, "mesh": cfg["desc"], "order": cfg["order"],
           "pde": "euler" if cfg["pde"] == 0 else "mhd_glm",
           "flux": {0: "rusanov", 1: "osher", 2: "rusanov_quadrature_free"}[flux]}
    if precisions is None:
        precisions = ((cw.FP32_MIXED, "fp32_mixed", steps), (cw.FP64, "fp64", max(3, steps // 2)))
    solvers = {}
    for prec, key, k in precisions:
        s = cw.Solver(m, cfg["order"], cfg["pde"], prec, stream=stream.cuda_stream, flux=flux)
        ms, kern_ms, _ = time_solver(s, stream, barrier, Q0, k)
        fp32 = prec == cw.FP32_MIXED
        alg = algorithmic(cfg["dim"], cfg["order"], cfg["pde"], fp32=fp32, flux=flux)
        kern, dom = kernel_rooflines(kern_ms, {"rec": mesh.nc, "flux": s.nf, "update": mesh.nc}, alg, pk, fp32)
        res[key] = {"value": mesh.nc / (ms / 1e3), "unit": "cell-updates/s", "ms_per_step": ms, "steps": k,
                    "kernels": kern, "roofline": roofline_line(kern, dom, pk, fp32, None)}
        solvers[key] = s
    if "fp32_mixed" in solvers and "fp64" in solvers:
        res["accuracy"] = accuracy_pair(solvers, mesh, Q0)
    for s in solvers.values():
        s.close()
    return res


def ale_mesh(wl, dim, n):
    """The ALE explosion's mesh: [-1, 1]^d, transmissive, n x n x 2 jittered
    triangles (2D) or n^3 x 6 jittered tetrahedra (3D)."""
    if dim == 2:
        return wl.tri_mesh(n, lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=False, jitter=0.2, seed=1234)
    return wl.tet_mesh(n, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), periodic=False, jitter=0.15, seed=1234)


ALE_ORDER = {2: 4, 3: 3}


def ale_oracle_rate(dim=2, n=None, steps=3, order=None):
    """The FP64 oracle's direct ALE step timed on the host (one thread) on a
    bounded sample of the same workload family: 40 x 40 x 2 triangles (3,200,
    the size of the paper's 2D Sedov mesh) or 6^3 x 6 tetrahedra (1,296), one
    untimed step first."""
    import oracle
    from paper_1612_09335_gb300 import workloads as wl
    n = n or (40 if dim == 2 else 6)
    mesh = ale_mesh(wl, dim, n)
    Q = wl.explosion_averages(mesh, sub=4)
    o = oracle.Oracle(mesh, order or ALE_ORDER[dim])
    Q, _ = o.ale_step(Q, o.stable_dt(Q))
    t0 = time.perf_counter()
    for _ in range(steps):
        Q, _ = o.ale_step(Q, o.stable_dt(Q))
    el = time.perf_counter() - t0
    shape = f"{n}x{n}x2 triangles" if dim == 2 else f"{n}^3x6 tetrahedra"
    return {"value": mesh.nc * steps / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{mesh.nc} cells ({shape}, same family), {steps} ALE steps after one untimed step, "
                      "single host thread"}


ALE_STAGES = ("geometry_and_least_squares", "reconstruction", "predictor", "nodal_solver", "faces", "update",
              "cfl_bound")


def ale_stages(s, steps):
    """Per-stage device time of `steps` further moving-mesh steps (CUDA events
    around each stage on the solver's stream, a pass of its own so that the
    timed steps carry no events): mean ms per step and share of the stages'
    sum."""
    s.profile(True)
    for _ in range(steps):
        s.step(0.0)
    ms, n = s.profile_read_stages(len(ALE_STAGES))
    s.profile(False)
    tot = sum(ms) or 1.0
    return {k: {"ms": ms[q] / max(1, n[q]), "share": ms[q] / tot} for q, k in enumerate(ALE_STAGES) if n[q]}


def ale_rate(cw, stream, barrier, dim=2, n=None, steps=None, warm=3, order=None):
    """Moving mesh: direct ALE steps (mesh velocity = fluid velocity) of the
    explosion (Sec. 3.2's ALE explosion, Table efficiency), Rusanov, on a
    transmissive mesh of [-1, 1]^d: 2D fourth order (M = 3) on n x n x 2
    triangles, 3D third order (M = 2) on n^3 x 6 tetrahedra; FP64 and
    FP32-mixed; CUDA events on the solver stream, device CFL step.  Accuracy
    of FP32-mixed against FP64 after `steps` steps of the FP64 solver's CFL
    step sizes (state and vertices), and its drift of sum |T| Q."""
    import dataclasses
    import numpy as np
    import torch
    from paper_1612_09335_gb300 import workloads as wl
    n = n or (256 if dim == 2 else 63)
    steps = steps or (10 if dim == 2 else 4)
    order = order or ALE_ORDER[dim]
    mesh = ale_mesh(wl, dim, n)
    Q0 = wl.explosion_averages(mesh, sub=4)
    m = cw.Mesh.from_workload(mesh)
    shape = f"{n}x{n}x2 triangles, jitter 20 %" if dim == 2 else f"{n}^3x6 tetrahedra, jitter 15 %"
    paper = ("2D, 17,340 triangles, reports tau_E = 6.6e-4 s" if dim == 2 else
             "3D, 1,469,472 tetrahedra, reports tau_E = 1.9e-2 s")
    out = {"cells": mesh.nc, "mesh": f"[-1,1]^{dim}, {shape}, transmissive, moving with the flow",
           "order": order,
           "note": f"the paper's ALE explosion ({paper} per element update on its CPU, Table efficiency): "
                   "context, not a target"}
    solvers = {}
    for prec, key in ((cw.FP32_MIXED, "fp32_mixed"), (cw.FP64, "fp64")):
        s = cw.Solver(m, order, 0, prec, stream=stream.cuda_stream, mesh_motion=cw.MOTION_LAGRANGE)
        s.set_state(Q0)
        for _ in range(warm):
            s.step(0.0)
        s.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(steps):
            s.step(0.0)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        s.sync()
        moved = float(abs(s.get_vertices() - mesh.xyz).max())
        v = mesh.nc * steps / (ms / 1e3)
        out[key] = {"value": v, "unit": "cell-updates/s", "ms_per_step": ms / steps, "steps": steps,
                    "max_vertex_displacement": moved, "tau_E_s": 1.0 / v,
                    "stages": ale_stages(s, steps)}
        solvers[key] = s
    for sv in solvers.values():
        sv.close()
    # accuracy on fresh solvers (the timed ones moved their meshes)
    a = cw.Solver(m, order, 0, cw.FP32_MIXED, stream=stream.cuda_stream, mesh_motion=cw.MOTION_LAGRANGE)
    b = cw.Solver(m, order, 0, cw.FP64, stream=stream.cuda_stream, mesh_motion=cw.MOTION_LAGRANGE)
    a.set_state(Q0)
    b.set_state(Q0)
    # the FP64 solver takes its device CFL step (the flow accelerates, so a
    # step fixed at t = 0 would outgrow the CFL bound); FP32-mixed follows
    # with the same step sizes
    dts = []
    for _ in range(steps):
        t0 = b.time()
        b.step(0.0)
        dts.append(b.time() - t0)
        a.step(dts[-1])
    dt = float(np.mean(dts))
    qa, qb = a.get_state(), b.get_state()
    xa, xb = a.get_vertices(), b.get_vertices()
    acc = accuracy_metrics(dataclasses.replace(mesh, xyz=xb), Q0, qa, qb)
    X0 = mesh.cell_vertices()
    v0 = np.abs(np.linalg.det(X0[:, 1:] - X0[:, :1])) / math.factorial(dim)
    Xa = dataclasses.replace(mesh, xyz=xa).cell_vertices()
    va = np.abs(np.linalg.det(Xa[:, 1:] - Xa[:, :1])) / math.factorial(dim)
    tot0 = v0 @ Q0
    scale = np.maximum(np.maximum(np.abs(tot0), v0 @ np.abs(Q0)), 1e-300)
    acc["conservation_drift_rel"] = [float(x) for x in np.abs(va @ qa - tot0) / np.maximum(scale, 1e-6 * scale.max())]
    acc.update({"reference": "FP64 moving-mesh step (parity-tested against the FP64 oracle's ALE step)",
                "steps": steps, "dt_mean": dt, "vertices_max_abs_diff": float(np.abs(xa - xb).max())})
    out["accuracy"] = acc
    a.close()
    b.close()
    m.close()
    return out


# ---------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1612_09335_gb300 import binding as cw

    if args.only_ale:
        st = torch.cuda.Stream()
        torch.cuda.set_stream(st)
        print(json.dumps({"ale": ale_rate(cw, st, torch.cuda.synchronize, dim=args.ale_dim, n=args.n,
                                          steps=args.steps, warm=args.warmup, order=args.ale_order)}))
        return
    name = args.workload
    cfg = WORKLOADS[name]
    mesh, Q0 = make_inputs(name, args.n)
    N = mesh.nc
    # a dedicated (non-default) stream: the library launches on it and the
    # CUDA events below are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    m = cw.Mesh.from_workload(mesh)
    s = cw.Solver(m, cfg["order"], cfg["pde"], cw.FP32_MIXED, stream=stream.cuda_stream)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    s.set_state(Q0)
    for _ in range(args.warmup):
        s.step(0.0)
    s.sync()
    s.set_state(Q0)
    s.profile(True)
    clk = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        s.step(0.0)
    e1.record(stream)
    barrier()
    t1 = time.perf_counter()
    clk.stop()
    ms = e0.elapsed_time(e1)
    kms, kn = s.profile_read()
    s.profile(False)
    s.sync()
    sim_time = s.time()
    ms = max_over_ranks(ms)
    value = replica_rate(ws, N, args.steps, ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    r_bytes = 4 * (mcal(cfg["order"] - 1, cfg["dim"]) - 1) * (cfg["dim"] * mcal(cfg["order"] - 1, cfg["dim"]) - 1) * N
    out["config"] = {"workload": name, "mesh": WORKLOADS[name]["desc"] if args.n is None else f"n={args.n}",
                     "cells": N, "faces": s.nf, "order": cfg["order"],
                     "pde": "euler" if cfg["pde"] == 0 else "mhd_glm", "dim": cfg["dim"],
                     "precision": "fp32_mixed (FP32 arithmetic; FP64 setup, FP64 cell-average accumulator)",
                     "time_step": "CFL bound computed on the device every step",
                     "l2": f"inputs larger than L2 (reconstruction matrices {r_bytes / 1e6:.0f} MB)",
                     "parallelism": f"replicas x{ws}", "simulated_time": sim_time}
    out["config"]["scheme"] = ("the paper's fixed-mesh ADER-CWENO step plus the positivity safeguard "
                               "(scaling limiter, face-point and predictor fallbacks; inactive on smooth data)")
    # measured FMA peaks of this device (FP32, FP64), clocks sampled meanwhile
    clk2 = ClockSampler(local)
    time.sleep(0.2)
    tp0 = time.perf_counter()
    fma32 = max(cw.cweno_measure_fma_peak(False)[0] for _ in range(3))
    fma64 = max(cw.cweno_measure_fma_peak(True)[0] for _ in range(3))
    tp1 = time.perf_counter()
    clk2.stop()
    pclk = clk2.summary(tp0, tp1)
    pk = peaks({"fp32_tflops": fma32, "fp64_tflops": fma64, "sm_mhz": pclk["sm_mhz"]})
    out["peaks"] = {"hbm_gbs": pk["hbm_gbs"], "hbm_src": pk["hbm_src"], "fp32_fma_tflops": fma32,
                    "fp64_fma_tflops": fma64, "sm_count": pk["sm_count"], "clocks": pclk,
                    "how": "cweno_measure_fma_peak: 16 independent FMA chains per thread, all SMs filled, "
                           "CUDA events, best of 3"}
    # per-kernel rooflines of the timed region
    names = ("k_rec_pred", "k_flux", "k_update")
    kern_ms = {names[q]: kms[q] / kn[q] for q in range(3) if kn[q]}
    alg = algorithmic(cfg["dim"], cfg["order"], cfg["pde"], fp32=True)
    kernels, dom = kernel_rooflines(kern_ms, {"rec": N, "flux": s.nf, "update": N}, alg, pk, True)
    out["roofline"] = roofline_line(kernels, dom, pk, True, measured_traffic(dom, name))
    step_bytes = sum(kernels[k]["bytes_per_unit"] * kernels[k]["units"] for k in kernels)
    out["step_hbm_frac"] = step_bytes / (ms / args.steps / 1e3) / 1e9 / pk["hbm_gbs"]
    out["kernels"] = kernels
    out["gpu_launches"] = int(sum(kn))
    out["clocks"] = clk.summary(t0, t1)
    solvers = {"fp32_mixed": s}
    # FP64 mode, same workload (the other precision of the metric)
    if not args.no_fp64:
        s64 = cw.Solver(m, cfg["order"], cfg["pde"], cw.FP64, stream=stream.cuda_stream)
        k64 = max(3, min(args.steps, 20))
        ms64, kern64_ms, _ = time_solver(s64, stream, barrier, Q0, k64, warm=1)
        alg64 = algorithmic(cfg["dim"], cfg["order"], cfg["pde"], fp32=False)
        kern64, dom64 = kernel_rooflines(kern64_ms, {"rec": N, "flux": s64.nf, "update": N}, alg64, pk, False)
        ms64 = max_over_ranks(ms64)
        out["fp64"] = {"value": ws * N / (ms64 / 1e3), "unit": "cell-updates/s", "steps": k64,
                       "ms_per_step": ms64, "kernels": kern64,
                       "roofline": roofline_line(kern64, dom64, pk, False, None)}
        solvers["fp64"] = s64
    # end to end through the C ABI with pinned host buffers
    if not args.no_e2e:
        nv = s.nv
        hin = torch.empty((N, nv), dtype=torch.float64, pin_memory=True)
        hin.numpy()[:] = Q0
        hout = torch.empty((N, nv), dtype=torch.float64, pin_memory=True)
        ke = max(3, min(args.steps, 30))
        s.set_state(hin)
        s.step(0.0)
        s.get_state(hout)
        barrier()
        ta = time.perf_counter()
        for _ in range(ke):
            s.set_state(hin)
            s.step(0.0)
            s.get_state(hout)
        barrier()
        tb = time.perf_counter()
        el = max_over_ranks(tb - ta)
        out["e2e"] = {"value": replica_rate(ws, N, ke, el), "unit": "cell-updates/s", "h2d_bytes_per_step": N * nv * 8,
                      "d2h_bytes_per_step": N * nv * 8, "steps": ke,
                      "path": "cweno_set_state(pinned host) + ader_cweno_step + cweno_get_state(pinned host)"}
    # accuracy of the FP32-mixed mode against the FP64 mode, and conservation
    if not args.no_accuracy and "fp64" in solvers:
        out["accuracy"] = accuracy_pair(solvers, mesh, Q0)
    for sv in solvers.values():
        sv.close()
    if rank == 0 and not args.no_serve:
        out["serving"] = serving_run(cw, args.serve_requests)
    if not args.no_other:
        out["other_workloads"] = {}
        for other in ("densitywave3d_p2", "orszagtang2d_p3", "explosion2d_p4", "densitywave3d_p4"):
            if other == name:
                continue
            out["other_workloads"][other] = workload_rate(cw, other, stream, barrier, pk, steps=10)
        # the other face fluxes on the bench workload
        out["flux_variants"] = {}
        for key, fl in (("osher", cw.FLUX_OSHER), ("rusanov_quadrature_free", cw.FLUX_RUSANOV_QF)):
            if fl == cw.FLUX_OSHER and cfg["pde"] != 0:
                continue
            out["flux_variants"][key] = workload_rate(cw, name, stream, barrier, pk, steps=20, flux=fl,
                                                      inputs=(mesh, Q0))
        # moving mesh (direct ALE), rank 0's GPU
        out["ale_explosion2d_p3"] = ale_rate(cw, stream, barrier)
        out["ale_explosion3d_p2"] = ale_rate(cw, stream, barrier, dim=3)
        # the paper's order for its moving-mesh tests (M = 3)
        out["ale_explosion3d_p3"] = ale_rate(cw, stream, barrier, dim=3, order=4, steps=3, warm=2)
        if rank == 0 and not args.no_cpu_baseline:
            out["ale_explosion2d_p3"]["cpu_baseline"] = ale_oracle_rate()
            out["ale_explosion3d_p2"]["cpu_baseline"] = ale_oracle_rate(dim=3, steps=2)
            out["ale_explosion3d_p3"]["cpu_baseline"] = ale_oracle_rate(dim=3, steps=1, order=4)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_run(name, cw=cw)
        out["accuracy_vs_oracle"] = out["cpu_baseline"].pop("vs_oracle")
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    name = args.workload
    cfg = WORKLOADS[name]
    oracle.build()
    nproc = os.cpu_count() or 1
    per_cell = {(2, 4, 0): 200e-6, (2, 3, 0): 65e-6, (3, 3, 0): 400e-6, (2, 4, 1): 900e-6}.get(
        (cfg["dim"], cfg["order"], cfg["pde"]), 300e-6)
    budget = min(5.0, 150.0 / max(1, args.steps + args.warmup))  # seconds of oracle work per step
    cells = max(256 * nproc, int(budget * nproc / per_cell))
    n = max(8, int(math.sqrt(cells / 2))) if cfg["dim"] == 2 else max(4, int(round((cells / 6) ** (1 / 3))))
    v, cores, nc, el = oracle_parallel_run(name, n, steps=args.steps, warmup=args.warmup, nproc=nproc)
    out = {"metric": METRIC, "value": v, "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": name, "cells": nc, "order": cfg["order"],
                      "pde": "euler" if cfg["pde"] == 0 else "mhd_glm", "dim": cfg["dim"],
                      "precision": "fp64 (oracle)"},
           "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                            "sample": f"{nc}-cell mesh of the same workload family per step (bounded sample), "
                                      f"{cores} worker processes each stepping a contiguous share of the cells"},
           "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="explosion2d_p3", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=None, help="mesh resolution override (small profiling cases)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the 3D, MHD and fifth-order workloads, the flux variants and the moving mesh")
    ap.add_argument("--ale-dim", type=int, default=2, choices=[2, 3], help="with --only-ale: 2D or 3D explosion")
    ap.add_argument("--ale-order", type=int, default=None, choices=[2, 3, 4], help="with --only-ale: order")
    ap.add_argument("--only-ale", action="store_true",
                    help="time only the moving-mesh (direct ALE) explosion; --n sets its resolution")
    ap.add_argument("--serve-requests", type=int, default=512,
                    help="requests in the serving mix (the full mix has 512)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
