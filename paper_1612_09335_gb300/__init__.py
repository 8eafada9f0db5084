"""GB300 ADER-CWENO: the fixed-mesh ADER-CWENO finite-volume step of
arXiv 1612.09335 as hand-written sm_103a CUDA behind a C ABI (include/cweno.h).

Importing the package loads nothing; ``build()`` compiles libcweno.so and
``binding`` wraps it.  ``workloads`` produces seeded synthetic inputs.
"""
from ._build import build  # noqa: F401

__all__ = ["build", "binding", "workloads"]
