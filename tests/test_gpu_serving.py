"""Serving loop (serve_create / serve_submit / serve_poll) on the GPU:
continuous batching of independent solves.  Each result must equal the same
solve run alone through the solver API, bitwise (no cross-request
reductions; same kernels, same inputs)."""
import time

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


def mix(wl, nreq=10, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nreq):
        n = int(rng.integers(8, 40))
        order = int(rng.integers(2, 5))
        mesh = wl.tri_mesh(n, periodic=True, jitter=0.2, seed=100 + k)
        if k % 2:
            Q = wl.cell_averages(mesh, lambda x: wl.vortex(x, eps=float(rng.uniform(1, 5))), n=4)
        else:
            Q = wl.explosion_averages(mesh, r0=0.3, centre=(0.5, 0.5), p_in=1.0, sub=4)
        out.append((mesh, Q, order))
    return out


def test_served_results_equal_alone(cw, wl):
    reqs = mix(wl)
    srv = cw.Server(max_slots=4)
    ids = [srv.submit(m, Q, order, 0.5, 15) for m, Q, order in reqs]
    srv.drain(300)
    got = []
    for rid in ids:
        st, Q, lat = srv.poll(rid)
        assert st == cw.REQ_DONE and Q is not None and lat > 0, srv.errors
        got.append(Q)
    stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["peak_running"] <= 4
    assert stats["cell_updates"] == sum(m.nc * 15 for m, _, _ in reqs)
    srv.close()
    for (m, Q0, order), Qs in zip(reqs, got):
        s = cw.Solver(cw.Mesh.from_workload(m), order, cw.EULER, cw.FP32_MIXED, cfl=0.5)
        s.set_state(Q0)
        s.run(15)
        s.sync()
        assert np.array_equal(s.get_state(), Qs)


def test_admission_by_memory_budget(cw, wl):
    """Six equal requests under a budget of 2.5 footprints: never all admitted
    at once, all complete; a request larger than the budget is refused."""
    reqs = []
    for k in range(6):
        m = wl.tri_mesh(30, seed=300 + k)
        reqs.append((m, wl.cell_averages(m, lambda x: wl.vortex(x), n=3), 4))
    probe = cw.Solver(cw.Mesh.from_workload(reqs[0][0]), 4, cw.EULER, cw.FP32_MIXED)
    budget = int(probe.footprint() * 2.5)
    probe.close()
    srv = cw.Server(mem_budget=budget, max_slots=16)
    ids = [srv.submit(m, Q, order, 0.5, 5) for m, Q, order in reqs]
    srv.drain(300)
    assert all(srv.poll(r)[0] == cw.REQ_DONE for r in ids)
    assert 1 <= srv.stats()["peak_running"] <= 2
    huge = wl.tri_mesh(300)
    with pytest.raises(cw.CwenoError) as e:
        srv.submit(huge, np.ones((huge.nc, 4)) * np.array([1, 0, 0, 2.5]), 4, 0.5, 5)
    assert e.value.code == cw.EBUSY
    srv.close()


def test_bad_request_fails_alone(cw, wl):
    good = mix(wl, nreq=3, seed=7)
    bad_mesh = wl.tri_mesh(10)
    bad_mesh.cells = bad_mesh.cells.copy()
    bad_mesh.cells[4] = bad_mesh.cells[4][[0, 2, 1]]  # clockwise cell
    srv = cw.Server(max_slots=2)
    ids = [srv.submit(m, Q, o, 0.5, 5) for m, Q, o in good[:2]]
    bad = srv.submit(bad_mesh, np.tile([1.0, 0, 0, 2.5], (bad_mesh.nc, 1)), 3, 0.5, 5)
    ids.append(srv.submit(*good[2][:2], good[2][2], 0.5, 5))
    srv.drain(300)
    assert srv.poll(bad)[0] == cw.REQ_ERROR
    assert all(srv.poll(r)[0] == cw.REQ_DONE for r in ids)
    srv.close()


def test_requests_overlap_on_device(cw, wl):
    """Many small requests admitted together finish faster than one after
    another through the same server with a single slot."""
    reqs = [(wl.tri_mesh(24, seed=200 + k), None, 3) for k in range(12)]
    reqs = [(m, wl.cell_averages(m, lambda x: wl.vortex(x), n=3), o) for m, _, o in reqs]

    def run(slots):
        srv = cw.Server(max_slots=slots)
        t0 = time.perf_counter()
        ids = [srv.submit(m, Q, o, 0.5, 40) for m, Q, o in reqs]
        srv.drain(300)
        el = time.perf_counter() - t0
        assert all(srv.poll(r)[0] == cw.REQ_DONE for r in ids)
        assert srv.stats()["peak_running"] <= slots
        srv.close()
        return el
    run(8)  # warm-up (reference tables, kernels)
    assert run(8) < run(1)


def test_zero_step_and_fifth_order_requests(cw, wl):
    """A request of zero steps returns its initial state unchanged; a
    fifth-order request is served like the others (same result as alone)."""
    m = wl.tri_mesh(20, seed=401)
    Q = wl.cell_averages(m, lambda x: wl.vortex(x), n=3)
    srv = cw.Server(max_slots=4)
    a = srv.submit(m, Q, 3, 0.5, 0)
    b = srv.submit(m, Q, 5, 0.5, 10)
    srv.drain(300)
    st, Qa, _ = srv.poll(a)
    assert st == cw.REQ_DONE and np.array_equal(Qa, Q)
    st, Qb, _ = srv.poll(b)
    assert st == cw.REQ_DONE, srv.errors
    srv.close()
    s = cw.Solver(cw.Mesh.from_workload(m), 5, cw.EULER, cw.FP32_MIXED, cfl=0.5)
    s.set_state(Q)
    s.run(10)
    s.sync()
    assert np.array_equal(s.get_state(), Qb)


def test_mixed_orders_submitted_mid_run_are_batched_and_equal_alone(cw, wl):
    """Requests of three orders, half submitted while the first half is
    already stepping: every result equals the same solve run alone through
    the solver API, bit for bit, and the steps were packed (each batched
    launch sequence advanced several requests on average)."""
    first = mix(wl, nreq=8, seed=11)
    second = mix(wl, nreq=8, seed=12)
    srv = cw.Server(max_slots=16)
    ids = [srv.submit(m, Q, order, 0.5, 30) for m, Q, order in first]
    t0 = time.perf_counter()
    while srv.stats()["ticks"] == 0 and time.perf_counter() - t0 < 120:
        time.sleep(0.002)
    assert srv.stats()["ticks"] > 0
    ids += [srv.submit(m, Q, order, 0.5, 20) for m, Q, order in second]
    srv.drain(300)
    got = []
    for rid in ids:
        st, Q, _ = srv.poll(rid)
        assert st == cw.REQ_DONE, srv.errors
        got.append(Q)
    stats = srv.stats()
    srv.close()
    assert stats["member_steps"] == 8 * 30 + 8 * 20
    assert stats["member_steps"] >= 2 * stats["ticks"]
    for (m, Q0, order), steps, Qs in zip(first + second, [30] * 8 + [20] * 8, got):
        s = cw.Solver(cw.Mesh.from_workload(m), order, cw.EULER, cw.FP32_MIXED, cfl=0.5)
        s.set_state(Q0)
        s.run(steps)
        s.sync()
        assert np.array_equal(s.get_state(), Qs)
