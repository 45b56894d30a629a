"""Builds libbysdf.so in-tree with nvcc for sm_103a (no CMake, no torch)."""
from __future__ import annotations

import os
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(PKG, "libbysdf.so")
# The index-checking build (-DBYSDF_DEBUG_BOUNDS): every checked index that
# falls out of range sets bit 2 of the launch's error word and is clamped;
# a separate library, built on demand by the tests that use it.
BOUNDS_BUILD_DIR = os.path.join(BUILD_DIR, "bounds")
BOUNDS_LIB_PATH = os.path.join(PKG, "libbysdf_bounds.so")
SOURCES = ["bysdf_api.cu", "bysdf_fwd.cu", "bysdf_fwd_eval.cu", "bysdf_fwd_sample.cu",
           "bysdf_fwd_pdf.cu", "bysdf_fwd_fused.cu", "bysdf_fwd_stoch.cu", "bysdf_bwd.cu",
           "bysdf_trace.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
# The forward, backward and ray-yarn kernels divide and take square roots
# with the hardware's approximate instructions (a few ulp: far inside the
# 1e-4 tolerance of values and gradients, and inside the margins of the
# tracer's conservative culling bounds), and flush single-precision
# denormals (below 2^-126) to zero, which spares those instructions their
# denormal scaling.
FAST_FLAGS = {s: ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
              for s in ("bysdf_fwd_eval.cu", "bysdf_fwd_sample.cu", "bysdf_fwd_pdf.cu",
                        "bysdf_fwd_fused.cu", "bysdf_fwd_stoch.cu", "bysdf_fwd.cu",
                        "bysdf_bwd.cu", "bysdf_trace.cu")}
_lock = threading.Lock()


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return [os.path.join(CSRC, s) for s in SOURCES] + hdrs + [os.path.join(INCLUDE, "bysdf.h")]


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          bounds: bool = False) -> str:
    """Compile the CUDA sources in parallel and link libbysdf.so (static
    cudart), or with bounds the index-checking libbysdf_bounds.so."""
    lib = BOUNDS_LIB_PATH if bounds else LIB_PATH
    bdir = BOUNDS_BUILD_DIR if bounds else BUILD_DIR
    defs = ["-DBYSDF_DEBUG_BOUNDS"] if bounds else []
    with _lock:
        if not force and not _stale(lib):
            return lib
        os.makedirs(bdir, exist_ok=True)
        nvcc = _nvcc()
        extra = ["-Xptxas", "-v"] if ptxas_info else []

        def compile_one(src):
            obj = os.path.join(bdir, src.replace(".cu", ".o"))
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, *FAST_FLAGS.get(src, []), *extra, "-c",
                   os.path.join(CSRC, src), "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
            if verbose or ptxas_info:
                sys.stderr.write(r.stderr)
            return obj

        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(compile_one, SOURCES))
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
        return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                bounds="--bounds" in sys.argv))
