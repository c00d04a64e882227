"""In-tree build of the CUDA library ``_build/liblbm.so`` for sm_103a.

Six translation units compiled in parallel with nvcc, linked against the
shared CUDA runtime (the same one PyTorch loads):
  lbm_api.cu    C ABI, initial state, read-back, finalisation (-fmad=false)
  step_f64.cu   FP64 fused step (-fmad=false: no contracted multiply-adds)
  step_lp.cu    FP32-arithmetic fused steps (FP32, FP16 and BF16 storage)
  geometry.cpp  host-side eye builder and mask validation
  noalloc.cu    observables with library-held device scratch
  vortex.cu     vortex intensity and centres (-fmad=false)
Host code is built with -ffp-contract=off so that the geometry builder's
floating-point decisions do not depend on the host architecture.
"""
from __future__ import annotations

import fcntl
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
          "-I", INCLUDE, "-I", CSRC]
UNITS = [
    ("lbm_api.cu", ["-fmad=false"]),
    ("step_f64.cu", ["-fmad=false"]),
    ("step_lp.cu", []),
    ("geometry.cpp", []),
    ("noalloc.cu", []),
    ("vortex.cu", ["-fmad=false"]),
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(INCLUDE, "lbm.h"))
    return out


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if a source is newer than it; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    with open(os.path.join(OUT_DIR, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        if not force and not stale():
            return LIB
        nvcc = _nvcc()

        def compile_unit(unit):
            name, extra = unit
            obj = os.path.join(OUT_DIR, name + ".o")
            cmd = [nvcc, *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, name), "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            subprocess.run(cmd, check=True)
            return obj

        with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
            objs = list(ex.map(compile_unit, UNITS))
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
