"""Builds libsnn.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit is compiled in parallel, then linked into one
shared library with the CUDA runtime linked statically.  Host code is compiled
without floating-point contraction, and device code with -fmad=false, so that
the FP32 path is reproducible bit for bit.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libsnn.so")
# the checked variant (-DSNN_CHECK): device bounds checks on the hot path's
# indexed writes, which set an error bit instead of writing out of bounds
LIB_CHECK = os.path.join(PKG, "libsnn_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["snn_api.cu", "build_kernels.cu", "step_kernels.cu", "persistent_kernels.cu", "persistent_tiled.cu", "persistent_owned.cu", "persistent_pull.cu", "shard_kernels.cu", "stdp_kernels.cu", "cdf_static.cu", "server.cu", "autotune.cu", "batch_kernels.cu"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsnn.so")


def _paths(check):
    """(library, object directory, flag stamp) of the release or checked variant."""
    if check:
        return LIB_CHECK, os.path.join(BUILD, "check"), os.path.join(BUILD, "check", "flags.txt")
    return LIB, BUILD, os.path.join(BUILD, "flags.txt")


def _user_flags():
    """Extra nvcc flags from SNN_NVCC_FLAGS (tuning macros such as
    -DSNN_DELIVER_UNROLL=8); a change of them forces a rebuild."""
    return os.environ.get("SNN_NVCC_FLAGS", "").split()


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false",
                   "-Xcompiler", "-fPIC,-ffp-contract=off,-O2,-fvisibility=hidden",
                   "-I", INCLUDE, "-I", CSRC, *_user_flags(), *extra]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "snn.h"))
    return files


def stale(check: bool = False) -> bool:
    lib, _, stamp = _paths(check)
    if not os.path.exists(lib):
        return True
    try:
        with open(stamp) as f:
            if f.read() != " ".join(_user_flags()):
                return True
    except OSError:
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, check: bool = False) -> str:
    """Build libsnn.so (or, with check=True, the checked libsnn_check.so)."""
    LIB, BUILD, STAMP = _paths(check)
    if not force and not stale(check):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DSNN_CHECK"] if check else [])

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose or ptxas_info:
            sys.stderr.write(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(" ".join(_user_flags()))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
