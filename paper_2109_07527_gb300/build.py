"""Build libcrmc.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into
``paper_2109_07527_gb300/libcrmc.so``.  No CPU fallback is built.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcrmc.so")
SOURCES = ["crmc_phase.cu", "crmc_md.cu", "crmc_api.cu", "crmc_noalloc.cu", "crmc_train.cu", "crmc_state.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "crmc.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _nvcc():
    for p in ("nvcc", "/usr/local/cuda/bin/nvcc"):
        try:
            subprocess.check_output([p, "--version"])
            return p
        except (OSError, subprocess.CalledProcessError):
            continue
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcrmc.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
