"""In-tree build of the CUDA library ``_build/liblbm.so`` for sm_103a.

Each translation unit under ``csrc/`` is compiled by its own ``nvcc -c`` in
parallel, then linked into one shared library that exports the C ABI of
``include/lbm.h``.  The CUDA runtime is linked statically, so the library
loads on a machine without a GPU (calls then fail with LBM_E_CUDA).
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm.so")
HEADER = os.path.join(ROOT, "include", "lbm.h")
SOURCES = ["stream_collide.cu", "kernels.cu", "runtime.cu", "static_scratch.cu", "adjoint.cu"]
# the cell kernels are compiled without implicit multiply-add contraction: a
# cell's arithmetic then rounds the same in every kernel that runs it (launch
# shapes, batched ensembles, the boundary kernel); the wanted FMAs are explicit
NO_CONTRACT = {"stream_collide.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile the library if a source or header is newer than it."""
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [HEADER, os.path.join(CSRC, "lbm_internal.cuh")]
    nvcc = _nvcc()
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            fmad = ["-fmad=false"] if src in NO_CONTRACT else []
            cmd = [nvcc, *ARCH, *FLAGS, *fmad, *extra_flags, "-c", s, "-o", o]
            jobs.append(cmd)
    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
