"""In-tree build of the CUDA library (sm_103a only).  No CPU fallback exists: the binding refuses to
load when the library is missing."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libkiops.so")
INCLUDE = os.path.join(ROOT, "include")
SOURCES = ["kiops_kernels_f64.cu", "kiops_kernels_f64_wide.cu", "kiops_kernels_f32.cu", "kiops_server.cu",
           "kiops_capi.cu", "kiops_integrate.cu", "kiops_probe.cu", "kiops_kernels_tma.cu",
           "kiops_kernels_tma_fixed.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "kiops.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + f".{os.getpid()}.o")
        cmd = [nvcc, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        return obj

    objs = [os.path.join(BUILD, os.path.splitext(src)[0] + f".{os.getpid()}.o") for src in SOURCES]
    try:
        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            list(ex.map(compile_one, SOURCES))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB
