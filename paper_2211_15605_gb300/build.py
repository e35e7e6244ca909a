"""Build libmppic in-tree for sm_103a with nvcc (no cmake, one translation unit)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmppic.so")
SOURCES = [os.path.join(CSRC, "mppic.cu")]
# the benchmark's FP64-rate probe: a separate small library, not part of the step's ABI
PROBE_SRC = os.path.join(CSRC, "probe.cu")
PROBE_LIB = os.path.join(OUT_DIR, "libmppic_probe.so")
DEPS = SOURCES + [os.path.join(CSRC, "mppic_device.cuh"), os.path.join(CSRC, "mppic_adjoint.cuh"),
               os.path.join(CSRC, "mppic_sort.cuh"), os.path.join(CSRC, "mppic_resort.cuh"), os.path.join(ROOT, "include", "mppic.h")]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-gencode", "arch=compute_103a,code=sm_103a",
              "-Xcompiler", "-fPIC", "-shared"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(lib, deps):
    return not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(p) for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libmppic (and the benchmark's probe library) for sm_103a, in parallel."""
    os.makedirs(OUT_DIR, exist_ok=True)
    jobs = []
    for lib, srcs, deps in ((LIB, SOURCES, DEPS), (PROBE_LIB, [PROBE_SRC], [PROBE_SRC])):
        if force or _stale(lib, deps):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [nvcc()] + NVCC_FLAGS + ["-o", tmp] + srcs
            if verbose:
                print(" ".join(cmd))
            jobs.append((subprocess.Popen(cmd), tmp, lib))
    failed = None
    for proc, tmp, lib in jobs:
        if proc.wait() != 0:
            failed = lib
        else:
            os.replace(tmp, lib)
    if failed:
        raise RuntimeError(f"nvcc failed building {failed}")
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
