"""Builds libmgm.so in-tree from csrc/*.cu for sm_103a (nvcc, one -gencode, files in parallel).

Setup translation units are compiled with --fmad=false so that every floating-point operation is
the one written in the source (bit-reproducible integer decisions and FP64 setup values); the
V-cycle and Krylov units keep fused multiply-add contraction.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libmgm.so")
BUILD = os.path.join(HERE, "_build")

EXACT = ["util", "knn", "knn_noalloc", "stencil", "coarsen", "order", "transfer", "hierarchy"]
FAST = ["vcycle", "gs_stream", "tail", "krylov", "multi", "learned", "eigs", "pattern", "capi"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")] + [os.path.join(INCLUDE, "mgm.h")]
    jobs = []
    for name in EXACT + FAST:
        src = os.path.join(CSRC, name + ".cu")
        obj = os.path.join(BUILD, name + ".o")
        if force or _stale(obj, [src] + headers):
            flags = [nvcc, ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                     "--fmad=" + ("false" if name in EXACT else "true"), "-c", src, "-o", obj]
            jobs.append(flags)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(BUILD, n + ".o") for n in EXACT + FAST]
    if force or jobs or _stale(OUT, objs):
        tmp = OUT + f".tmp{os.getpid()}"
        run([nvcc, ARCH, "-shared", "-o", tmp] + objs)
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
