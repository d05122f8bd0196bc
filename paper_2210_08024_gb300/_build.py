"""Builds the in-tree CUDA library libtc_gb300.so for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel and linked into one shared
library next to this file; the Python binding loads it with ctypes.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtc_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["tc_api.cu", "tc_onezone.cu", "tc_sixray.cu", "tc_pdr.cu", "tc_order.cu", "tc_k_paper.cu", "tc_k_newton.cu", "tc_k_mixed.cu", "tc_mlp.cu", "tc_peak.cu",
           "tc_static.cu", "tc_k_seeded3.cu", "tc_k_seeded4.cu", "tc_k_newton_coop.cu", "tc_k_mixed_coop.cu",
           "tc_df64_diag.cu"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def _flags():
    return ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"] + ARCH


# The mixed-precision step kernels evaluate their Newton iterations on FP32 source terms
# and correct every root with a high-precision polish, so their FP32 arithmetic may use
# the fast approximate intrinsics (exp, log, divide; flush-to-zero).  This changes no
# FP64 operation, and the df64 arithmetic of the polish (tc_df64.cuh) uses rounded
# intrinsics for its error-free transformations and corrects its FP32 first
# approximations.  Measured on the 128^3 slab (with an FP64 polish): mixed 250 -> 215 ms,
# mixed + seed 295 -> 238 ms, with the same iteration counts and the same parity results.
# tc_df64_diag.cu holds the device check of the df64 arithmetic, built the same way.
# tc_order.cu predicts each cell's cost class from FP32 source terms (its FP64 kernel,
# k_rates, is untouched by the option).
FAST_FP32 = {"tc_k_mixed.cu", "tc_k_seeded3.cu", "tc_k_mixed_coop.cu", "tc_df64_diag.cu", "tc_order.cu"}


def _compile(src: str) -> tuple[str, str]:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    extra = ["--use_fast_math"] if src in FAST_FP32 else []
    cmd = [nvcc()] + _flags() + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s" % (src, r.stderr[-4000:]))
    return obj, r.stderr


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    inc = os.path.join(os.path.dirname(HERE), "include")
    deps += [os.path.join(inc, f) for f in os.listdir(inc)]
    deps.append(__file__)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        res = list(ex.map(_compile, srcs))
    log = "\n".join(r[1] for r in res)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        fh.write(log)
    if verbose:
        print(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc(), "-shared", "-cudart", "shared"] + ARCH + [r[0] for r in res] + ["-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr[-4000:])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
    print(LIB)
