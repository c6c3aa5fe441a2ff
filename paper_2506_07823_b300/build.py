"""Build ``libpdilqr.so`` (CUDA, sm_103a) in-tree with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libpdilqr.so")
SOURCES = ["pdilqr.cu", "serve.cu", "ops_small.cu", "ops_12.cu", "ops_24.cu", "ops_36.cu",
           "ops_48.cu", "ops_96.cu", "ops_192.cu", "peaks.cu"]
BUILD_DIR = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files


def _compile(nvcc, src, obj, verbose):
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "-I" + INCLUDE, "-c", "-o", obj, src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    return obj


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile the translation units that are out of date (in parallel) and
    link libpdilqr.so.  A unit is recompiled when its object is older than the
    unit itself or than any header (headers are shared by every unit)."""
    from concurrent.futures import ThreadPoolExecutor
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(BUILD_DIR, exist_ok=True)
    jobs = [(os.path.join(CSRC, src), os.path.join(BUILD_DIR, src.replace(".cu", ".o")))
            for src in SOURCES]
    headers = max(os.path.getmtime(f) for f in _inputs() if not f.endswith(".cu"))

    def fresh(src, obj):
        return (not force and os.path.exists(obj) and
                os.path.getmtime(obj) >= max(os.path.getmtime(src), headers))

    todo = [j for j in jobs if not fresh(*j)]
    objs = [j[1] for j in jobs]
    if not todo and os.path.exists(LIB) and \
            os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs):
        return LIB
    with ThreadPoolExecutor(max_workers=max(1, len(todo))) as ex:
        list(ex.map(lambda j: _compile(nvcc, j[0], j[1], verbose), todo))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose="-v" in sys.argv)
