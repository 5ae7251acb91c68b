"""Builds the sm_103a shared library libarcher_epid.so in-tree with nvcc.

The library is the product's compute path; no Python fallback exists, so a
missing or stale build is an error at import time of the binding.
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
LIB = PKG / "libarcher_epid.so"
SOURCES = ["mc_api.cu", "mc_transport.cu", "mc_aux.cu", "mc_noalloc.cu", "physics_tables.cpp", "dn_kernels.cu",
           "dn_api.cu"]
HEADERS = ["mc_device.cuh", "mc_aux.h", "physics_tables.h", "dn_tc.cuh", "dn_kernels.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = [CSRC / s for s in SOURCES + HEADERS] + [INCLUDE / "archer_epid.h", INCLUDE / "archer_denoise.h"]
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> Path:
    if not force and not stale():
        return LIB
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           f"-I{INCLUDE}", "-o", str(tmp), *[str(CSRC / s) for s in SOURCES]]
    if verbose_ptxas:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)
