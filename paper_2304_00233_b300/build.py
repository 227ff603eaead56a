"""Build libemm.so (CUDA kernels + C ABI) in-tree for sm_103a.

    python -m paper_2304_00233_b300.build [--force] [-v]

Compiles ``csrc/emm_kernels.cu``, ``csrc/emm_adjoint.cu``, ``csrc/emm_model.cu``,
``csrc/emm_graph.cu`` and ``csrc/emm_setup.cpp`` with nvcc into
``paper_2304_00233_b300/libemm.so`` (the shared library the Python binding and
any C caller load).  Host code is compiled without FMA contraction so that
the FP64 setup tables are reproducible."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libemm.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("emm_kernels.cu", "emm_adjoint.cu", "emm_model.cu", "emm_graph.cu", "emm_setup.cpp")]
HEADERS = [os.path.join(HERE, "csrc", "emm_internal.h"), os.path.join(HERE, "csrc", "emm_tma.cuh"),
           os.path.join(os.path.dirname(HERE), "include", "emm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libemm")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in SOURCES + HEADERS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-shared",
           "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
           "-o", tmp, *SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
