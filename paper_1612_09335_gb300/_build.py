"""Build the CUDA library libcweno.so in-tree (nvcc, sm_103a only).

Translation units compile in parallel; the shared library is linked with the
static CUDA runtime.  Nothing here falls back to anything: a missing nvcc or
a failed compile raises.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libcweno.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["kern_euler2.cu", "kern_euler3.cu", "kern_euler3_p4.cu", "kern_euler3_p4f.cu", "kern_mhd2.cu", "api.cu", "noalloc.cu", "setup_gpu.cu", "lsq_gpu.cu", "ale.cu", "peak.cu"]
# per-file flags: the device stencil search keeps the host's FP64 arithmetic
# (no FMA contraction), so that its distance keys and cone tests agree
CU_FLAGS = {"setup_gpu.cu": ["--fmad=false"]}
CPP_SOURCES = ["refelem.cpp", "mesh.cpp", "setup.cpp", "serve.cpp"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcweno")
    return p


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "cweno.h"))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def _compile(src: str, extra: list[str], objdir: str = OBJ) -> str:
    nvcc = _nvcc()
    obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-Xptxas", "-O3", *CU_FLAGS.get(src, []), *extra, "-c", path, "-o", obj]
    else:
        cmd = [nvcc, "-O2", "-std=c++17", "-x", "c++", "-Xcompiler", "-fPIC,-ffp-contract=off",
               *extra, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, extra: list[str] | None = None,
          out: str | None = None) -> str:
    """Compile and link; `out` (with `extra` flags) builds a variant library
    elsewhere, objects beside it."""
    lib = out or LIB
    objdir = OBJ if out is None else os.path.join(os.path.dirname(os.path.abspath(out)), "obj")
    if not force and up_to_date(lib):
        return lib
    os.makedirs(objdir, exist_ok=True)
    os.makedirs(os.path.dirname(os.path.abspath(lib)), exist_ok=True)
    extra = list(extra or [])
    srcs = CU_SOURCES + CPP_SOURCES
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, objdir), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [_nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None)
