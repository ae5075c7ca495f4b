"""Compiles libgj.so (CUDA, sm_103a) in-tree with nvcc, and its checked
build libgj_checks.so (the same sources with -DGJ_CHECKS: device bounds
checks that report GJ_E_CHECK instead of faulting).

Each ``csrc/*.cu`` file is compiled to an object under ``_build/`` (the
checked objects under ``_build/checks/``) and the objects are linked into
``paper_1802_03760_b300/libgj.so`` and ``libgj_checks.so``. Only changed
sources are recompiled. Run ``python -m paper_1802_03760_b300.build``.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libgj.so")
LIB_CHECKS = os.path.join(HERE, "libgj_checks.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src: str, verbose: bool, checks: bool = False) -> str:
    obj = os.path.join(BUILD, "checks" if checks else "", os.path.basename(src) + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _headers_mtime()):
        return obj
    cmd = [NVCC] + ARCH + FLAGS + (["-DGJ_CHECKS"] if checks else []) + (["-Xptxas", "-v"] if verbose else []) + \
        ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def _link(lib: str, objs) -> None:
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)


def build(verbose: bool = False, checks: bool = True) -> str:
    """Builds libgj.so and (checks=True) libgj_checks.so; returns libgj.so's path."""
    os.makedirs(os.path.join(BUILD, "checks"), exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = [(s, False) for s in srcs] + ([(s, True) for s in srcs] if checks else [])
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(16, len(jobs))) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], verbose, j[1]), jobs))
    _link(LIB, objs[:len(srcs)])
    if checks:
        _link(LIB_CHECKS, objs[len(srcs):])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
