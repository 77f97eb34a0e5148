"""Build libmpnl.so (the C ABI of include/mpnl.h) for sm_103a with nvcc.

Each .cu file is compiled in parallel to an object under ``_build/`` and the
objects are linked into ``paper_2409_14355_gb300/libmpnl.so`` (in-tree, not
installed); the benchmark's FP32 FMA probe (``bench/``) goes into a library
of its own, ``libmpnl_bench.so``.  ``python -m paper_2409_14355_gb300.build [-v]`` rebuilds it;
``-v`` also prints ptxas register / shared-memory usage.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmpnl.so")
# the benchmark's measurement helpers, kept out of the detector's library
BENCH_SRC = os.path.join(PKG, "bench")
BENCH_LIB = os.path.join(PKG, "libmpnl_bench.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no multiply-add is contracted behind the source's back; the
# kernels write every FMA they want explicitly (fmaf).  So the arithmetic of
# a function does not depend on the context it is inlined into, and a unit
# gives bit-identical results from the per-call and the batch kernels.
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
         "--expt-relaxed-constexpr", "-fmad=false"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def bench_sources() -> list[str]:
    return sorted(os.path.join(BENCH_SRC, f) for f in os.listdir(BENCH_SRC) if f.endswith(".cu"))


def _deps() -> list[str]:
    out = [os.path.join(INCLUDE, "mpnl.h")]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return out


def _stale(target: str, inputs: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(p) > t for p in inputs)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    nvcc = _nvcc()
    deps = _deps()
    jobs = []
    objs, bench_objs = [], []
    for src in sources() + bench_sources():
        obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
        (bench_objs if os.path.dirname(src) == BENCH_SRC else objs).append(obj)
        if force or verbose or _stale(obj, [src] + deps):
            cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
            if verbose:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    for lib, ob in ((LIB, objs), (BENCH_LIB, bench_objs)):
        if force or jobs or _stale(lib, ob):
            tmp = lib + f".tmp{os.getpid()}"
            subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *ob], check=True)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    build(force="-f" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
