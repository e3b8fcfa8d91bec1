"""Build the hdmd CUDA library in-tree for GB300 (sm_103a).

Compiles each translation unit of ``csrc/`` with nvcc in parallel and links
``_lib/libhdmd.so`` (static CUDA runtime, C ABI of ``include/hdmd.h``).
Objects go to ``_build/``; both folders are git-ignored.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIB_DIR, "libhdmd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["kernels_bin.cu", "kernels_nbr.cu", "kernels_force.cu", "kernels_swap.cu",
         "kernels_batch_d2.cu", "kernels_batch_d4.cu", "kernels_batch_d6.cu",
         "kernels_batch_d8.cu", "kernels_batch_d9.cu", "system.cu",
         "batch.cu", "noalloc.cu", "kernels_obs.cu", "kernels_resident.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the hdmd CUDA library cannot be built")


def _newest_input() -> float:
    paths = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    paths.append(os.path.join(ROOT, "include", "hdmd.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include")] + list(extra_flags)

    def compile_one(unit):
        obj = os.path.join(OBJ, unit.replace(".cu", ".o"))
        cmd = [cc] + flags + ["-c", os.path.join(SRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
