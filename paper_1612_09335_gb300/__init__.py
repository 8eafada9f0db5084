"""GB300 ADER-CWENO: the fixed-mesh ADER-CWENO finite-volume step of
arXiv 1612.09335, and its direct ALE step on moving triangle and tetrahedron
meshes, as hand-written sm_103a CUDA behind a C ABI (include/cweno.h).

    from paper_1612_09335_gb300 import binding as cw, workloads as wl
    mesh, Q = wl.vortex_2d(64)
    s = cw.Solver(cw.Mesh.from_workload(mesh), 4, cw.EULER, cw.FP32_MIXED)
    s.set_state(Q); s.run(100); Q1 = s.get_state()
    # moving mesh (mesh velocity = fluid velocity), FP64
    a = cw.Solver(cw.Mesh.from_workload(mesh), 4, cw.EULER, cw.FP64, mesh_motion=cw.MOTION_LAGRANGE)
    a.set_state(Q); a.run(10); xyz = a.get_vertices()

Importing the package loads nothing; ``build()`` compiles libcweno.so and
``binding`` wraps it.  ``workloads`` produces seeded synthetic inputs.
"""
from ._build import build  # noqa: F401

__all__ = ["build", "binding", "workloads"]
