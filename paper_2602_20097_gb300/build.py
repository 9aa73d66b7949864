"""Build ``libqai.so`` in-tree: one nvcc compile per translation unit, in
parallel, for sm_103a only, then a shared-library link.

``python -m paper_2602_20097_gb300.build`` (or ``build()``) recompiles when a
source or header is newer than the library. ``QAI_PTXAS_VERBOSE=1`` adds
``-Xptxas -v`` (registers, spills, shared memory per kernel).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libqai.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the qai CUDA library cannot be built")
    return path


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + [os.path.join(ROOT, "include", "qai.h")])


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def flags():
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")] + ARCH
    if os.environ.get("QAI_PTXAS_VERBOSE"):
        f += ["-Xptxas", "-v"]
    return f


def build(force: bool = False, verbose: bool = False) -> str:
    with _lock:
        if not force and not stale():
            return LIB
        objdir = os.path.join(LIBDIR, "obj")
        os.makedirs(objdir, exist_ok=True)
        cc = nvcc()

        def compile_one(src):
            obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
            cmd = [cc, "-c", src, "-o", obj] + flags()
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
            if verbose and r.stderr:
                sys.stderr.write(r.stderr)
            return obj

        with cf.ThreadPoolExecutor(max_workers=max(1, len(sources()))) as ex:
            objs = list(ex.map(compile_one, sources()))
        tmp = LIB + f".tmp{os.getpid()}"
        r = subprocess.run([cc, "-shared", "-o", tmp] + objs + ARCH, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
