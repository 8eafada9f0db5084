"""Checkpoint / resume through the C ABI: the FP64 cell averages read after k
steps, given to a fresh solver of the same mesh, continue the run bit for
bit (the state is the whole state: in FP32-mixed mode set_state forms the
same FP32 hi/lo split the update does).  Fixed step lengths."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1612_09335_gb300 as pkg
    pkg.build()
    from paper_1612_09335_gb300 import binding
    return binding


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_continues_bit_for_bit(cw, prec):
    from paper_1612_09335_gb300 import workloads as wl
    mesh, Q = wl.vortex_2d(20)
    m = cw.Mesh.from_workload(mesh)
    dt = 0.002
    a = cw.Solver(m, 3, cw.EULER, prec)
    a.set_state(Q)
    for _ in range(6):
        a.step(dt)
    b = cw.Solver(m, 3, cw.EULER, prec)
    b.set_state(Q)
    for _ in range(3):
        b.step(dt)
    ckpt = b.get_state()
    b.close()
    c = cw.Solver(m, 3, cw.EULER, prec)
    c.set_state(ckpt)
    for _ in range(3):
        c.step(dt)
    assert np.array_equal(a.get_state(), c.get_state())
