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
           "dn_api.cu", "mc_probe.cu"]
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


# Per-source flags.  The FP32 transport is compiled with approximate
# division, square root and transcendentals (nvcc --use_fast_math: the
# hardware's approximate instructions, denormals flushed to zero); its
# parity with the FP64 oracle is tested at the same tolerances as with IEEE
# division.  Everything else (statistics, ray sums, the denoiser) keeps the
# default IEEE arithmetic.
EXTRA = {"mc_transport.cu": ["--use_fast_math"]}


def build(force: bool = False, verbose_ptxas: bool = False) -> Path:
    if not force and not stale():
        return LIB
    import tempfile
    base = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}"]
    if verbose_ptxas:
        base.append("-Xptxas=-v")
    with tempfile.TemporaryDirectory(prefix="archer_build_") as tmpdir:
        objs, procs = [], []
        for src in SOURCES:
            obj = os.path.join(tmpdir, src + ".o")
            objs.append(obj)
            procs.append(subprocess.Popen([*base, *EXTRA.get(src, []), "-c", str(CSRC / src), "-o", obj]))
        bad = [src for src, pr in zip(SOURCES, procs) if pr.wait() != 0]
        if bad:
            raise subprocess.CalledProcessError(1, f"nvcc {' '.join(bad)}")
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp.so")
        subprocess.run([_nvcc(), *ARCH, "-shared", "-o", str(tmp), *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)
