"""In-tree build of the decoder library (nvcc, sm_103a) and the workload helper (gcc)."""
from __future__ import annotations

import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB_PATH = os.path.join(PKG, "libngdbf.so")
SOURCES = [os.path.join(CSRC, f) for f in ("ngdbf_decode.cu", "ngdbf_multi.cu", "ngdbf_multi_cluster.cu",
                                           "ngdbf_server.cu", "ngdbf_plain.cu", "ngdbf_hostmem.cu")]
HEADERS = [os.path.join(CSRC, h) for h in ("ngdbf_device.cuh", "ngdbf_kernels.cuh", "ngdbf_multi.h", "ngdbf_host.h")]
DEPS = SOURCES + HEADERS + [os.path.join(ROOT, "include", "ngdbf.h")]

NVCC_FLAGS = [
    "-std=c++17", "-O3", "-lineinfo",
    "-gencode", "arch=compute_103a,code=sm_103a",
    # every FP32 operation of the method is an explicitly rounded intrinsic;
    # no contraction elsewhere either
    "--fmad=false",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
]

def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_cuda(force: bool = False, verbose: bool = False) -> str:
    """Compiles libngdbf.so next to this file (translation units in parallel); returns its path."""
    if force or stale(LIB_PATH, DEPS):
        tag = f"{os.getpid()}"
        objs = [f"{src}.{tag}.o" for src in SOURCES]
        procs = [subprocess.Popen([nvcc(), *NVCC_FLAGS, *(["-Xptxas", "-v"] if verbose else []),
                                   "-c", "-o", obj, src]) for src, obj in zip(SOURCES, objs)]
        codes = [p.wait() for p in procs]
        try:
            if any(codes):
                raise subprocess.CalledProcessError(max(codes), "nvcc -c")
            tmp = f"{LIB_PATH}.{tag}.tmp"
            subprocess.check_call([nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a",
                                   "-o", tmp, *objs])
            os.replace(tmp, LIB_PATH)
        finally:
            for o in objs:
                if os.path.exists(o):
                    os.remove(o)
    return LIB_PATH


def build_all(force: bool = False) -> None:
    from . import workload
    workload.build(force)
    build_cuda(force)
