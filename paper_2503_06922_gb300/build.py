"""Builds libaccfem.so (the C-ABI library of the hot path) in-tree for sm_103a with nvcc.

Each CUDA translation unit is compiled in parallel, then linked into a shared library next to
this file.  ``python -m paper_2503_06922_gb300.build`` or ``build()`` from Python.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libaccfem.so")
UNITS = ["element", "collide", "segment", "btd", "contact", "primal", "update", "api", "batch", "serve", "noalloc"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no implicit contraction of a * b + c into a fused multiply-add; every FMA of the
# kernels is an explicit fma() in the source, so the rounding of each expression is fixed by the
# source alone (the same block body gives the same bits in its single-instance and batched kernels,
# and the collision predicates round like a plain FP64 evaluation).
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _compile(unit, objdir):
    src = os.path.join(CSRC, unit + ".cu")
    obj = os.path.join(objdir, unit + ".o")
    cmd = [_nvcc()] + ARCH + FLAGS + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, " ".join(cmd), r.stderr))
    return obj


def build(verbose=False):
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(u, objdir), UNITS))
    cmd = [_nvcc()] + ARCH + ["-shared", "-o", OUT] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    if verbose:
        print("built", OUT)
    return OUT


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
