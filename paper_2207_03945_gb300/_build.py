"""Builds the CUDA library libflock.so in-tree with nvcc for sm_103a."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libflock.so")
SOURCES = ["flock.cu", "flock_batch.cu", "flock_rollout.cu", "flock_nvtx.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no FMA contraction anywhere (the model's FP32 formulas are
# written with explicit round-to-nearest intrinsics as well); IEEE division
# and square root; denormals kept.
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
         "-ftz=false", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


LIB_DEBUG = os.path.join(HERE, "libflock_debug.so")
# the debug build: every FLOCK_DEBUG check on (index bounds that latch
# FLOCK_ERR_BOUNDS and skip the access; device code still never traps)
DEBUG_FLAGS = ["-DFLOCK_DEBUG=1"]


def _jobs(nvcc, headers, debug, force, verbose):
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    os.makedirs(bdir, exist_ok=True)
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [nvcc] + ARCH + FLAGS + (DEBUG_FLAGS if debug else []) + ["-c", s, "-o", o]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    return objs, jobs


def build(force: bool = False, verbose: bool = False, debug: bool = True) -> str:
    """Compiles libflock.so (and, with debug, libflock_debug.so, the same
    sources with FLOCK_DEBUG checks) with nvcc, all translation units in
    parallel.  Returns the path of libflock.so."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "flock.h"))
    nvcc = _nvcc()
    targets = [(LIB, False)] + ([(LIB_DEBUG, True)] if debug else [])
    plan = []
    jobs = []
    for lib, dbg in targets:
        objs, js = _jobs(nvcc, headers, dbg, force, verbose)
        plan.append((lib, objs, bool(js)))
        jobs += js
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for r in ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs):
            if r.returncode != 0:
                raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
            if verbose:
                print(r.stderr)
    for lib, objs, rebuilt in plan:
        if force or rebuilt or _stale(lib, objs):
            tmp = lib + ".tmp%d" % os.getpid()
            subprocess.run([nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs,
                           check=True, capture_output=True)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
