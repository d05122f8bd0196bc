"""FP64 work per cell of the library's step, for the roofline of the benchmark.

Builds and runs csrc/tc_workcount.cu, a host build of the library's own step
functions with counting hooks.  It writes work_slab128.json: for each mode, the FP64
operations per cell by class (add, mul, div, sqrt, exp, log) of one step of dt = 1e4 yr
on a seeded sample of the 128^3 slab.  bench.py weights them by the FMA-slot cost of
each class, measured in the same run, to state the work one launch performs.

The dense 3x3 linear algebra of each Newton iteration (FD-Jacobian differencing, the
residual, Gaussian elimination, damping and convergence test) is not templated on the
scalar type; its counts per iteration are stated here from the code:
    FP64 Newton iteration   63 add, 55 mul, 16 div   (one division per Jacobian column)
    FP64 chord iteration    42 add, 40 mul, 13 div   (the same without the differencing:
                                                      21 add, 15 mul, 9 div)
    mixed Newton iteration  18 add, 12 mul,  6 div   (its FP64 part: residual, damped step
                                                      and test; the correction is solved in FP32)
    polish iteration        16 add, 12 mul,  6 div   (the same, residual from df64 sources)
    paper-scheme substep    18 add, 18 mul,  8 div   (FD slope, T update, 2x2 solve)
    predictor sweep         30 add, 30 mul,  8 div   (2x2 closed form, T step, change)

The mixed mode's high-precision evaluations run in df64 (double-float, csrc/tc_df64.cuh)
on the FP32 pipes.  Their operations by class are counted the same way ("mode2_df64");
each costs this many FP32-pipe instructions, counted from tc_df64.cuh (error-free
transformations included; exp and log with their call overhead):
    add 11, mul 7, div 28, sqrt 20, exp 125, log 170

    python -m paper_2210_08024_gb300.work               # count, write work_slab128.json
    python -m paper_2210_08024_gb300.work --breakdown   # FP64 slots per building block
"""
from __future__ import annotations

import json
import os
import shutil
import subprocess
import sys
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "work_slab128.json")
LINALG = {
    "newton64_it": {"add": 63, "mul": 55, "div": 16},
    "chord64_it": {"add": 42, "mul": 40, "div": 13},
    "newton32_it": {"add": 18, "mul": 12, "div": 6},
    "polish_it": {"add": 16, "mul": 12, "div": 6},
    "substep_paper": {"add": 18, "mul": 18, "div": 8},
    "picard_it": {"add": 30, "mul": 30, "div": 8},
}
DF64_FP32_INST = {"add": 11, "mul": 7, "div": 28, "sqrt": 20, "exp": 125, "log": 170}
CLASSES = ("add", "mul", "div", "sqrt", "exp", "log")
BLOCKS = {"chem_T": "cost_chem_T", "cool_T": "cost_cool_T", "temp_step": "cost_temp_step", "source": "cost_source",
          "equil": "cost_equil_setup", "equil_it": "cost_equil_iter", "dust": "cost_dust_setup",
          "dust_it": "cost_dust_iter"}


def build(tmp: str) -> str:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = os.path.join(tmp, "tc_workcount")
    cmd = [nvcc, "-std=c++17", "-O2", "-x", "cu", "-gencode", "arch=compute_103a,code=sm_103a",
           os.path.join(HERE, "csrc", "tc_workcount.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


def _ops(calls: dict, counts: dict, linalg: bool) -> dict:
    tot = {c: 0.0 for c in CLASSES}
    for blk, key in BLOCKS.items():
        for c in CLASSES:
            tot[c] += calls.get(blk, 0.0) * counts[key][c]
    if linalg:
        for blk, la in LINALG.items():
            for c, v in la.items():
                tot[c] += calls.get(blk, 0.0) * v
    return {c: round(v, 2) for c, v in tot.items()}


def per_cell(counts: dict) -> dict:
    """FP64 operations per cell by class for each mode; for the mixed mode also its FP32
    operations ("mode2_fp32": the same building blocks instantiated in FP32, whose
    exp, log, sqrt and divide the fast-math build issues to the MUFU pipe) and its df64
    operations ("mode2_df64", with "fp32_inst": their FP32-pipe instructions)."""
    out = {}
    for mode in ("mode0", "mode1", "mode2"):
        out[mode] = _ops(counts[mode]["fp64"], counts, True)
        out[mode]["substeps"] = counts[mode]["substeps"]
    out["mode2_fp32"] = _ops(counts["mode2"]["fp32"], counts, False)
    hp = _ops(counts["mode2"].get("df64", {}), counts, False)
    hp["fp32_inst"] = round(sum(hp[c] * DF64_FP32_INST[c] for c in CLASSES), 1)
    out["mode2_df64"] = hp
    return out


def algorithmic(counts: dict) -> dict:
    """The method's own work knobs per slab cell: substeps, evaluations of the source
    terms f (FP64, FP32 and df64 together, and the FP64 ones alone), Newton-type
    iterations per substep and polish corrections per substep."""
    out = {}
    for mode in ("mode0", "mode1", "mode2"):
        k, f, h = counts[mode]["fp64"], counts[mode]["fp32"], counts[mode].get("df64", {})
        ns = counts[mode]["substeps"]
        src = k["source"] + f["source"] + h.get("source", 0.0)
        its = k["newton64_it"] + k["chord64_it"] + k["newton32_it"]
        out[mode] = {"substeps": round(ns, 4), "source_evals": round(src, 3),
                     "source_evals_per_substep": round(src / ns, 3) if ns else 0.0,
                     "fp64_source_evals": round(k["source"], 3),
                     "iterations_per_substep": round(its / ns, 3) if ns else 0.0,
                     "polish_per_substep": round(k["polish_it"] / ns, 3) if ns else 0.0}
    return out


def main(sample: int = 8192):
    import synthgen
    c = synthgen.slab()
    idx = np.sort(np.random.default_rng(12345).choice(c["n"].size, sample, replace=False))
    sub = synthgen.subset(c, idx)
    keys = ("n", "chi_pe", "chi_lw", "f_h2", "f_c", "F_lyc", "xi", "Zg", "Zd", "T", "xH2", "xHp")
    with tempfile.TemporaryDirectory() as tmp:
        exe = build(tmp)
        path = os.path.join(tmp, "cells.bin")
        with open(path, "wb") as fh:
            fh.write(np.int64(sample).tobytes())
            for k in keys:
                fh.write(np.ascontiguousarray(np.broadcast_to(np.asarray(sub[k], np.float64), (sample,))).tobytes())
            fh.write(np.float64(synthgen.DT_1E4YR).tobytes())
        r = subprocess.run([exe, path], check=True, capture_output=True, text=True)
    counts = json.loads(r.stdout)
    res = {"_comment": "FP64 operations per cell of one step (dt = 1e4 yr) on %d seeded cells of the 128^3 slab, "
                       "counted from the library's own step functions (paper_2210_08024_gb300/work.py)." % sample,
           "per_cell": per_cell(counts), "algorithmic": algorithmic(counts), "raw": counts}
    with open(OUT, "w") as fh:
        json.dump(res, fh, indent=1)
    print(OUT)
    return res


# FMA-slot cost per operation class, as tc_peak measures it on a GB300 (the benchmark
# measures them again in each run; these are the values of one run, for the breakdown)
SLOT_WEIGHTS = {"add": 1.0, "mul": 1.0, "div": 5.67, "sqrt": 8.61, "exp": 16.0, "log": 30.2}


def breakdown(res: dict, mode: str = "mode1") -> list:
    """FP64 FMA slots per cell of one mode by building block (calls x cost per call, and
    the hand-counted dense algebra of each iteration), largest first: where the FP64
    work of the step goes."""
    raw = res["raw"]
    calls = raw[mode]["fp64"]
    rows = []
    for blk, key in BLOCKS.items():
        n = calls.get(blk, 0.0)
        rows.append((blk, n, n * sum(raw[key][c] * SLOT_WEIGHTS[c] for c in CLASSES)))
    for blk, la in LINALG.items():
        n = calls.get(blk, 0.0)
        rows.append((blk, n, n * sum(v * SLOT_WEIGHTS[c] for c, v in la.items())))
    rows = [r for r in rows if r[2] > 0.0]
    return sorted(rows, key=lambda r: -r[2])


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "--breakdown":
        with open(OUT) as fh:
            res = json.load(fh)
        for mode in ("mode1", "mode0"):
            rows = breakdown(res, mode)
            tot = sum(r[2] for r in rows)
            print("%s: %.0f FMA slots per cell" % (mode, tot))
            for blk, n, sl in rows:
                print("  %-12s %7.2f calls  %7.0f slots  %5.1f%%" % (blk, n, sl, 100.0 * sl / tot))
    else:
        main()
