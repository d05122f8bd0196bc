"""Benchmark of the thermochemistry source step (arXiv:2210.08024, Sec. 6.1) on GB300.

Workload: the 128^3 = 2,097,152-cell TIGRESS-like slab (lognormal density, two-phase
pressure relation, six-ray columns mapped to the FUV/LW fields, H2 self-shielding and
attenuated CR rate; see synthgen.slab), advanced by one step of dt = 1e4 yr.  One
benchmark step = one tc_step over every cell of the slab from the same initial state
(the state arrays are restored from a pristine device copy before each launch, inside
the timed region).  The inputs (~220 MB) exceed the 129 MB L2.

Metric: cell-updates per second.  `value` is the device-resident throughput of the
plain FP64 solver (coupled implicit backward Euler by Newton); `modes` lists every
mode measured in the same run.  `e2e` repeats the plain-FP64 measurement through the
host-buffer entry point tc_step_host (pinned host arrays; the H2D copy of the inputs
and the D2H copy of the results are inside the timed region).

--impl reference times the CPU oracle (the plain FP64 C++ statement of the method) on
the host cores on a bounded sample of the same workload.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under torchrun, each
rank advances its own slab (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthgen  # noqa: E402

DT = synthgen.DT_1E4YR
METRIC = "thermochemistry cell-updates/sec (1 GB300): plain FP64 vs MLP-seeded mixed at oracle tol"
UNIT = "cell-updates/s"
# Nominal FP64 rate of a GB300 (152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz ~ 1.26e12).
FP64_NOMINAL_TFLOPS = 1.25

STATE_KEYS = ("T", "xH2", "xHp")
# DRAM bytes per cell of one k_step<1> launch on the 128^3 slab in the benchmark's
# autotuned shape (64 threads x 1824 blocks, 768 resident threads per SM), from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass,
# profiles/k_step_fp64_slab128.md): 20.07 GB read + 29.21 GB written for 2,097,152
# cells.  Almost all of it is the per-thread stack (spills at the 80-register cap and
# the structs passed to the out-of-line physics): ~3 KB per thread for 768 resident
# threads per SM is ~350 MB, almost three times L2.  The cells' own data are 152 B.
TRAFFIC_BYTES_PER_CELL = 23499.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--side", type=int, default=128)
    ap.add_argument("--modes", default="newton,mixed,mixed_seeded,newton_seeded,paper",
                    help="comma list of modes to time (first = headline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-peaks", action="store_true", help="skip the pipe microbenchmarks (no roofline)")
    ap.add_argument("--configs", action="store_true",
                    help="instead of the benchmark line, time every workload config and its error vs the oracle")
    ap.add_argument("--no-drivers", action="store_true",
                    help="skip the one-zone, six-ray and PDR legs (timed after the step)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----- multi-rank host logic (one process per GPU; cells are independent, so each rank
# advances its own slab and the only collectives are the timing barrier and reduction)
def workload_key(rank: int) -> int:
    """Seed key of the slab a rank advances: every rank gets a different slab."""
    return 2 + rank


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """The largest x over the ranks: the job's time is its slowest rank's."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ncell_per_rank: int, ws: int, steps: int, ms: float) -> float:
    """Cell-updates per second of the whole job: every rank's cells over the slowest
    rank's time (weak scaling)."""
    return ws * ncell_per_rank * steps / (ms * 1e-3)


def work_per_cell():
    """FP64 operations per cell by class (add, mul, div, sqrt, exp, log) of one step on
    the slab, per mode (and the mixed mode's FP32 operations), counted from the library's
    own step functions (paper_2210_08024_gb300/work.py)."""
    path = os.path.join(ROOT, "paper_2210_08024_gb300", "work_slab128.json")
    with open(path) as fh:
        return json.load(fh)["per_cell"]


def algorithmic_per_cell():
    """Substeps, source-term evaluations and iterations per slab cell of each mode
    (the method's own work knobs, counted like work_per_cell)."""
    path = os.path.join(ROOT, "paper_2210_08024_gb300", "work_slab128.json")
    with open(path) as fh:
        return json.load(fh)["algorithmic"]


MODE_WORK = {"paper": "mode0", "newton": "mode1", "mixed": "mode2", "newton_seeded": "mode1", "mixed_seeded": "mode2"}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


def measure_peaks(tc, torch):
    """FP64 pipe rate and the FMA-slot cost of each FP64 operation class, measured with
    the library's microbenchmark kernels on this GPU."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    grid, block, iters = sms * 8, 256, 2048
    sink = torch.empty(grid * block, dtype=torch.float64, device="cuda")
    chains = tc.tc_peak_chains()
    st = torch.cuda.current_stream()
    rates = {}
    for name, kind, it in (("fma", 0, iters), ("exp", 2, iters // 16), ("log", 3, iters // 16),
                           ("sqrt", 4, iters // 8), ("div", 5, iters // 8), ("pow", 6, iters // 32),
                           ("fma32", 1, iters * 8), ("mufu", 8, iters * 2), ("df64_muladd", 9, iters),
                           ("df64_exp", 10, iters // 16)):
        tc.tc_peak_launch(kind, grid, block, it, sink)
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            tc.tc_peak_launch(kind, grid, block, it, sink)
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        rates[name] = grid * block * chains * it / (best * 1e-3)  # operations per second
    fma = rates["fma"]
    weights = {"add": 1.0, "mul": 1.0, "cmp": 0.0}
    for k in ("div", "sqrt", "exp", "log", "pow"):
        weights[k] = fma / rates[k]
    return {"fp64_fma_per_s": fma, "fp32_fma_per_s": rates["fma32"], "mufu_per_s": rates["mufu"], "rates": rates,
            "weights": weights,
            # df64 (double-float) operations against their FP64 counterparts on this GPU
            "df64_vs_fp64": {"muladd": rates["df64_muladd"] / fma, "exp": rates["df64_exp"] / rates["exp"]}}


def flops_per_cell(counts: dict, weights: dict) -> float:
    """FP64 work in FMA-equivalent flops: an add or a multiply is 1 flop; a divide,
    sqrt, exp or log costs its measured number of FMA slots at 2 flops per slot."""
    return counts["add"] + counts["mul"] + 2.0 * sum(counts[k] * weights[k] for k in ("div", "sqrt", "exp", "log"))


def run_gpu(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2210_08024_gb300 as P
    from paper_2210_08024_gb300 import tc

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    cells = synthgen.slab(side=args.side, key=workload_key(rank))
    ncell = int(cells["n"].size)
    dev = tc.to_device(cells)
    pristine = {k: dev[k].clone() for k in STATE_KEYS}
    stream = torch.cuda.current_stream()
    mode_ids = {"newton": tc.TC_MODE_NEWTON_FP64, "paper": tc.TC_MODE_PAPER_FP64, "mixed": tc.TC_MODE_MIXED,
                "newton_seeded": tc.TC_MODE_NEWTON_FP64_SEEDED, "mixed_seeded": tc.TC_MODE_MIXED_SEEDED}
    from paper_2210_08024_gb300 import seed_net
    blob = open(seed_net.DEFAULT_BLOB, "rb").read() if os.path.exists(seed_net.DEFAULT_BLOB) else None
    modes = [m for m in args.modes.split(",") if m and (blob is not None or "seeded" not in m)]
    peaks = measure_peaks(tc, torch) if (rank == 0 and not args.no_peaks) else None

    def restore():
        for k in STATE_KEYS:
            dev[k].copy_(pristine[k])

    results = {}
    clocks = None
    for mi, mname in enumerate(modes):
        st = tc.Stepper(mode_ids[mname])
        if "seeded" in mname:
            st.load_mlp(blob)
        f = tc.make_fields(dev)
        # launch shape: the library's autotuner times its candidates on this workload
        # (on a scratch copy of the initial state) before the timed region
        restore()
        shape = tc.tc_autotune(st.h, f, DT, stream)
        for _ in range(args.warmup):
            restore()
            tc.tc_step(st.h, f, DT, stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if mi == 0 else None
        if sampler:
            sampler.start()
        l0 = st.launches()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        t0.record(stream)
        for s in range(args.steps):
            restore()
            kev[s][0].record(stream)
            tc.tc_step(st.h, f, DT, stream)
            kev[s][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        if sampler:
            clocks = sampler.stop()
        ms = t0.elapsed_time(t1)
        kms = [a.elapsed_time(b) for a, b in kev]
        launches = st.launches() - l0
        ms = max_over_ranks(ms, ws, "cuda")
        nbad = tc.tc_sync_status(st.h, dev["status"])
        results[mname] = {"ms_per_step": ms / args.steps, "kernel_ms": float(np.mean(kms)),
                          "value": job_throughput(ncell, ws, args.steps, ms), "launches": launches,
                          "cells_not_ok": nbad, "newton_iters_per_cell": float(dev["iters"].double().mean().item()),
                          "launch_shape": shape, "mode_id": mode_ids[mname]}
        if "seeded" in mname:
            stt = dev["status"]
            results[mname]["cells_with_a_seeded_solve"] = float(((stt & tc.TC_ST_SEEDED) != 0).double().mean().item())
            results[mname]["cells_with_a_failed_seed"] = float(((stt & tc.TC_ST_SEED_FAIL) != 0).double().mean().item())
        st.close()

    head = modes[0]
    e2e = None if args.no_e2e else run_e2e(args, tc, torch, cells, ncell, mode_ids[head], stream, barrier, ws)
    hint = None if (args.no_drivers or rank != 0) else run_hint(args, tc, torch, stream, cells)
    drivers = None
    if rank == 0 and not args.no_drivers:
        drivers = {"onezone": run_onezone(args, tc, torch, stream), "sixray": run_sixray(args, tc, torch, stream, peaks),
                   "pdr": run_pdr(args, tc, torch, stream), "config1_latency": run_latency(args, tc, torch, stream)}
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return None
    out = report(args, results, head, ncell, peaks, e2e, clocks, cells, ws)
    out["drivers"] = drivers
    out["second_step_cost_hint"] = hint
    return out


def run_latency(args, tc, torch, stream):
    """The 4096 random states of config 1 (one step of 1e4 yr): a launch far too small to
    fill the GPU, whose time is the latency of its slowest cells.  Plain FP64 and mixed,
    one lane per cell against the warp-cooperative kernels (four lanes per cell, the
    library's automatic choice for this size)."""
    cells = synthgen.cells_4096()
    dev = tc.to_device(cells)
    pristine = {k: dev[k].clone() for k in STATE_KEYS}
    out = {"workload": "4096 random states (log n in [-2,4], log T in [1,7]), dt = 1e4 yr"}
    for mname, mode in (("newton", tc.TC_MODE_NEWTON_FP64), ("mixed", tc.TC_MODE_MIXED)):
        row = {}
        for lpc in (1, 4):
            st = tc.Stepper(mode, lanes_per_cell=lpc)
            f = tc.make_fields(dev)
            times = []
            for r in range(6):
                for k in STATE_KEYS:
                    dev[k].copy_(pristine[k])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                tc.tc_step(st.h, f, DT, stream)
                e1.record(stream)
                e1.synchronize()
                if r > 0:
                    times.append(e0.elapsed_time(e1))
            st.close()
            ms = float(np.median(times))
            row["lanes_per_cell_%d" % lpc] = {"ms": ms, "cell_updates_per_s": cells["n"].size / (ms * 1e-3)}
        row["speedup_4_over_1"] = row["lanes_per_cell_1"]["ms"] / row["lanes_per_cell_4"]["ms"]
        out[mname] = row
    return out


def run_hint(args, tc, torch, stream, cells):
    """A second step of the slab, from the state the first one produced, ordered either
    by the predicted substep count or by the first step's Newton iterations as a cost
    hint (tc_fields.cost_hint): what a simulation calling the library every step gets."""
    out = {}
    for mname, mode in (("newton", tc.TC_MODE_NEWTON_FP64), ("mixed", tc.TC_MODE_MIXED)):
        d = tc.to_device(cells)
        st = tc.Stepper(mode)
        st.step(d, DT, stream)
        torch.cuda.synchronize()
        start = {k: d[k].clone() for k in STATE_KEYS}
        prev_iters = d["iters"].clone()
        res = {}
        for name, hint in (("predicted", None), ("previous_step_iterations", prev_iters)):
            d["cost_hint"] = hint
            f = tc.make_fields(d)

            def call():
                for k in STATE_KEYS:
                    d[k].copy_(start[k])
                tc.tc_step(st.h, f, DT, stream)
            res[name] = _time_call(call, stream, 3)
        st.close()
        res["unit"] = "ms per step"
        out[mname] = res
    return out



def _time_call(fn, stream, reps, flush=None):
    """Median CUDA-event time (ms) of fn() on `stream` over `reps` calls after one
    warm-up; `flush` (a large tensor) is overwritten before each timed call."""
    import torch
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


# One-zone equilibrium curves (Sec. 7.1, Fig. f:minmax): 64 FUV intensities chi0 in
# [0.1, 1e3] (xi0 = 2e-16 chi0) x 4 metallicities Z' = Z'_g = Z'_d in {0.1, 0.3, 1, 3},
# 512 densities in [1e-2, 1e4] cm^-3, 1e2 Myr in 10 chunks, FP64 Newton, k_gr = 3e-17 Z'_d.
ONEZONE = dict(nchi=64, Z=(0.1, 0.3, 1.0, 3.0), nn=512, lo=-2.0, hi=4.0, t_end_myr=100.0, nchunk=10)


def onezone_grid():
    o = ONEZONE
    chi = np.logspace(-1, 3, o["nchi"])
    chi0 = np.repeat(chi, len(o["Z"]))
    Z = np.tile(np.array(o["Z"]), o["nchi"])
    return np.logspace(o["lo"], o["hi"], o["nn"]), chi0, 2e-16 * chi0, Z, Z


def run_onezone(args, tc, torch, stream):
    """Times tc_eq_curves on the Fig. f:minmax grid; the oracle's driver is timed on a
    seeded sample of 16 of its curves."""
    n_axis, chi0, xi0, Zg, Zd = onezone_grid()
    t_end = ONEZONE["t_end_myr"] * 1e6 * 3.15576e7
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64, flags=tc.TC_CONST_KGR)
    kw = dict(t_end_s=t_end, nchunk=ONEZONE["nchunk"])
    out = st.eq_curves(n_axis, chi0, xi0, Zg, Zd, stream=stream, **kw)
    l0 = st.launches()
    reps = max(1, min(args.steps, 3))
    ms = _time_call(lambda: st.eq_curves(n_axis, chi0, xi0, Zg, Zd, stream=stream, out=out, **kw), stream, reps)
    launches = (st.launches() - l0) // (reps + 1)
    st.close()
    ncell = n_axis.size * chi0.size
    res = {"workload": "%d curves (64 chi0 in [0.1, 1e3] x Z' in %s) x %d densities in [1e-2, 1e4] cm^-3, "
                       "1e2 Myr in %d chunks, FP64 Newton" % (chi0.size, list(ONEZONE["Z"]), n_axis.size,
                                                             ONEZONE["nchunk"]),
           "cells": ncell, "ms": ms, "cell_equilibria_per_s": ncell / (ms * 1e-3),
           "curves_per_s": chi0.size / (ms * 1e-3), "gpu_launches": launches,
           "cells_not_ok": int(((out["status"] & tc.TC_ST_ERROR_MASK) != 0).sum().item()),
           "curves_with_two_phases": int((out["i_min"] > 0).sum().item())}
    if not args.no_cpu_baseline:
        import oracle
        from oracle import onezone as oz
        pick = np.sort(np.random.default_rng(5).choice(chi0.size, 16, replace=False))
        a = time.perf_counter()
        oz.curves(n_axis, chi0[pick], xi0[pick], Zg[pick], Zd[pick],
                  oracle.default_params(mode=1, flags=oracle.F_CONST_KGR), t_end=t_end, nchunk=ONEZONE["nchunk"])
        el = time.perf_counter() - a
        res["cpu_baseline"] = {"value": pick.size * n_axis.size / el, "unit": "cell-equilibria/s",
                               "cores": os.cpu_count() or 1, "kind": "oracle",
                               "sample": "%d seeded curves of the grid (%d cells), %.1f s" %
                                         (pick.size, pick.size * n_axis.size, el)}
    return res


# FP64 operations per cell of tc_sixray, counted from the kernel source: per ray the
# H2 self-shielding factor (4 divides, a square root, an exponential), the ray weight
# (an exponential and a square root) and ~15 adds/multiplies with the scans; per cell
# the two cell averages (expm1 and a divide each), the two fields (an exponential each),
# f_shld,H2 and N_eff (a divide each, a logarithm), the CR rate and the two chi0/6 (a divide each).
SIXRAY_OPS = {"add": 50.0, "mul": 40.0, "div": 31.0, "sqrt": 12.0, "exp": 16.0, "log": 1.0}


def run_sixray(args, tc, torch, stream, peaks):
    """Times tc_sixray on the slab's densities and H2 fractions laid out on 128^3 and
    256^3 grids of 4 pc cells (L2 flushed before each call); the oracle is timed on the
    64^3 corner of the first."""
    res = {}
    dx = 4.0 * 3.0856775814913673e18
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for side in (128, 256):
        c = synthgen.slab(side=side, key=2)
        n = torch.from_numpy(np.ascontiguousarray(c["n"].reshape(side, side, side))).cuda()
        x = torch.from_numpy(np.array(np.broadcast_to(c["xH2"], c["n"].shape).reshape(side, side, side))).cuda()
        out = tc.tc_sixray(n, x, dx, stream=stream)
        ms = _time_call(lambda: tc.tc_sixray(n, x, dx, out=out, stream=stream), stream, max(3, args.steps), flush)
        ncell = side ** 3
        r = {"grid": "%d^3" % side, "cells": ncell, "ms": ms, "cells_per_s": ncell / (ms * 1e-3),
             "gpu_launches": 3, "l2": "flushed before each call"}
        if peaks is not None:
            fl = flops_per_cell(SIXRAY_OPS, peaks["weights"])
            ach = fl * ncell / (ms * 1e-3) / 1e12
            pk = 2.0 * peaks["fp64_fma_per_s"] / 1e12
            r["roofline"] = {"bound": "alu", "pipe": "fp64", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                             "frac": ach / pk, "work": "FP64 ops per cell counted from the kernels (%.0f flops)" % fl}
        res["%d" % side] = r
        del n, x, out
    del flush
    if not args.no_cpu_baseline:
        from oracle import sixray as osr
        c = synthgen.slab(side=128, key=2)
        n = c["n"].reshape(128, 128, 128)[:64, :64, :64].copy()
        x = np.broadcast_to(c["xH2"], c["n"].shape).reshape(128, 128, 128)[:64, :64, :64].copy()
        a = time.perf_counter()
        osr.sixray(n, x, dx)
        el = time.perf_counter() - a
        res["cpu_baseline"] = {"value": 64 ** 3 / el, "unit": "cells/s", "cores": 1, "kind": "oracle",
                               "sample": "64^3 corner of the 128^3 grid, numpy, %.2f s" % el}
    return res


def pdr_suite():
    """Sec. 7.3 suites, batched: n_H in 16 values over [10, 1e4] x chi0 in 16 values over
    [0.1, 1e4] x xi0 in {0, 2e-18, 2e-17, 2e-16} s^-1, keeping the slabs whose transition
    column the paper could resolve (more than three cells of >= 1e-3 pc); 100 cells per
    slab resolving the no-CR transition column by ~25 cells."""
    from oracle import pdr as opdr
    n, chi0, xi0 = (a.ravel() for a in np.meshgrid(np.logspace(1, 4, 16), np.logspace(-1, 4, 16),
                                                    [0.0, 2e-18, 2e-17, 2e-16], indexing="ij"))
    Nt = opdr.bialy_sternberg_ntrans(chi0, n)
    keep = Nt / n >= 3 * 1e-3 * 3.0856775814913673e18
    n, chi0, xi0, Nt = n[keep], chi0[keep], xi0[keep], Nt[keep]
    return n, chi0, xi0, Nt, Nt / 25.0 / n


def run_pdr(args, tc, torch, stream):
    """Times tc_pdr on the batched suites (3e2 Myr in 300 chunks, FP64 Newton); the
    oracle is timed on 8 of the slabs."""
    from oracle import pdr as opdr
    n, chi0, xi0, Nt, dx = pdr_suite()
    one = np.ones_like(n)
    t_end = 3e2 * 1e6 * 3.15576e7
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64, flags=tc.TC_CONST_KGR)
    out = st.pdr(n, chi0, xi0, one, dx, 100, stream=stream, t_end_s=t_end, nchunk=300)
    l0 = st.launches()
    ms = _time_call(lambda: st.pdr(n, chi0, xi0, one, dx, 100, stream=stream, out=out, t_end_s=t_end, nchunk=300),
                    stream, 1)
    launches = (st.launches() - l0) // 2
    st.close()
    nocr = xi0 == 0.0
    ratio = out["N_trans"].cpu().numpy()[nocr] / Nt[nocr]
    res = {"workload": "%d slabs x 100 cells (n 10..1e4, chi0 0.1..1e4, xi0 0..2e-16), 3e2 Myr in 300 chunks, "
                       "FP64 Newton" % n.size, "ms": ms, "slabs_per_s": n.size / (ms * 1e-3),
           "cell_chunks_per_s": n.size * 100 * 300 / (ms * 1e-3), "gpu_launches": launches,
           "cells_not_ok": int(((out["status"] & tc.TC_ST_ERROR_MASK) != 0).sum().item()),
           "N_trans_over_analytic_no_cr": {"min": float(ratio.min()), "max": float(ratio.max())}}
    if not args.no_cpu_baseline:
        import oracle
        pick = np.sort(np.random.default_rng(6).choice(n.size, 8, replace=False))
        a = time.perf_counter()
        opdr.slabs(n[pick], chi0[pick], xi0[pick], one[pick], dx[pick], 100,
                   oracle.default_params(mode=1, flags=oracle.F_CONST_KGR), t_end=t_end, nchunk=300)
        el = time.perf_counter() - a
        res["cpu_baseline"] = {"value": pick.size / el, "unit": "slabs/s", "cores": os.cpu_count() or 1,
                               "kind": "oracle", "sample": "8 seeded slabs of the suite, %.1f s" % el}
    return res


def run_e2e(args, tc, torch, cells, ncell, mode_id, stream, barrier, ws):
    """Same metric through the host-buffer entry point: pinned host arrays in, results
    out, copies inside the timed region."""
    host = {}
    for k in tc.INPUT_KEYS + STATE_KEYS:
        t = torch.empty(ncell, dtype=torch.float64, pin_memory=True)
        t.numpy()[:] = np.asarray(cells[k], dtype=np.float64)
        host[k] = t
    for k in ("xe", "xCp", "xCO"):
        host[k] = torch.zeros(ncell, dtype=torch.float64, pin_memory=True)
    for k in ("nsub", "status"):
        host[k] = torch.zeros(ncell, dtype=torch.int32, pin_memory=True)
    hf = tc.tc_fields()
    for cname, key in tc.FIELD_KEYS.items():
        setattr(hf, cname, host[key].data_ptr() if key in host else None)
    hf.ncell = ncell
    hf.Zg_val = 1.0
    hf.Zd_val = 1.0
    st = tc.Stepper(mode_id)
    h2d = sum(host[k].numel() * 8 for k in tc.INPUT_KEYS + STATE_KEYS)
    d2h = sum(host[k].numel() * host[k].element_size() for k in ("T", "xH2", "xHp", "xe", "xCp", "xCO", "nsub", "status"))
    pristine_host = {k: host[k].clone() for k in STATE_KEYS}
    for _ in range(max(1, args.warmup)):
        for k in STATE_KEYS:
            host[k].copy_(pristine_host[k])
        tc.tc_step_host(st.h, hf, DT, stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = 0.0
    for s in range(args.steps):
        for k in STATE_KEYS:
            host[k].copy_(pristine_host[k])
        a = time.perf_counter()
        tc.tc_step_host(st.h, hf, DT, stream)  # copies in, runs, copies out, synchronises
        e2e_ms += (time.perf_counter() - a) * 1e3
    barrier()
    e2e_ms = max_over_ranks(e2e_ms, ws, "cuda")
    st.close()
    return {"value": job_throughput(ncell, ws, args.steps, e2e_ms), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "api": "tc_step_host"}


def report(args, results, head, ncell, peaks, e2e, clocks, cells, ws):
    # roofline of the step kernel (FP64 pipe): the FP64 work of one launch (per-cell
    # counts of the library's own step, weighted by the FMA-slot cost of each operation
    # class measured in this run) over the CUDA-event duration of the launch.
    work = work_per_cell()
    algo = algorithmic_per_cell()
    r = results[head]
    roofline = None
    if peaks is not None:
        roofline = roofline_of(work, r, head, ncell, peaks)
        roofline["algorithmic_per_cell"] = algo[MODE_WORK[head]]
        for name, rr in results.items():
            rl = roofline_of(work, rr, name, ncell, peaks)
            rr["fp64_roofline_frac"] = rl["frac"]
            rr["fp64_tflops"] = rl["achieved"]
            rr["algorithmic_per_cell"] = algo[MODE_WORK[name]]
            if MODE_WORK[name] == "mode2":
                rr["fp32_pipes"] = fp32_fractions(work["mode2_fp32"], work["mode2_df64"], rr, ncell, peaks)
    cpu = None if args.no_cpu_baseline else cpu_baseline(cells, head)
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "slab%d: %d^3 = %d-cell TIGRESS-like slab, one step of dt = 1e4 yr" %
                                  (args.side, args.side, ncell),
                      "mode": head, "cells_per_gpu": ncell, "l2": "inputs larger than L2 (%.0f MB)" %
                      (ncell * 13 * 8 / 1e6), "parallelism": "dp%d (independent cells)" % ws},
           "modes": {k: {kk: vv for kk, vv in v.items() if kk != "mode_id"} for k, v in results.items()},
           "speedup_vs_plain_fp64": {k: v["value"] / results["newton"]["value"] for k, v in results.items()
                                     if "newton" in results},
           "gpu_launches": r["launches"], "e2e": e2e, "roofline": roofline, "clocks": clocks,
           "peaks": None if peaks is None else {
               "fp64_tflops": 2.0 * peaks["fp64_fma_per_s"] / 1e12,
               "fp32_tflops": 2.0 * peaks["fp32_fma_per_s"] / 1e12,
               "mufu_ops_per_s": peaks["mufu_per_s"],
               "df64_vs_fp64": peaks["df64_vs_fp64"],
               "fma_slot_weights": peaks["weights"]},
           "cpu_baseline": cpu}
    return out


def fp32_fractions(w32, w_df, r, ncell, peaks):
    """FP32 side of a mixed launch.  FP32 work: the FP32 evaluations' flops (add and
    multiply, plus the multiply that accompanies each approximate exp, log, sqrt and
    divide) and the df64 evaluations' FP32-pipe instructions (work_slab128.json,
    mode2_df64.fp32_inst: each df64 operation class times its instruction count),
    against the measured FP32 FMA issue rate (one instruction per lane and clock).  MUFU
    operations (one per exp, log, sqrt and divide of the fast-math FP32 evaluations)
    against the measured MUFU rate.  Counts per slab cell times the cells of the launch."""
    t = r["kernel_ms"] * 1e-3
    special = sum(w32[k] for k in ("div", "sqrt", "exp", "log"))
    inst = (w32["add"] + w32["mul"] + special + w_df["fp32_inst"]) * ncell
    mufu = special * ncell
    return {"fp32_inst_per_s": inst / t, "fp32_frac": inst / t / peaks["fp32_fma_per_s"],
            "df64_share_of_fp32_inst": w_df["fp32_inst"] / (w32["add"] + w32["mul"] + special + w_df["fp32_inst"]),
            "mufu_ops_per_s": mufu / t, "mufu_frac": mufu / t / peaks["mufu_per_s"],
            "work": "FP32 ops and df64 FP32 instructions per cell of the library's mixed step (work_slab128.json, "
                    "mode2_fp32, mode2_df64) x %d cells" % ncell}


def roofline_of(work, r, mode, ncell, peaks):
    fl = flops_per_cell(work[MODE_WORK[mode]], peaks["weights"]) * ncell
    achieved = fl / (r["kernel_ms"] * 1e-3) / 1e12
    peak = 2.0 * peaks["fp64_fma_per_s"] / 1e12
    return {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": (TRAFFIC_BYTES_PER_CELL * ncell
                                           if mode == "newton" and TRAFFIC_BYTES_PER_CELL else None),
            "peak_source": "measured FP64 FMA rate (library microbenchmark, this run); nominal %.2f" %
                           FP64_NOMINAL_TFLOPS,
            "work": "FP64 flops of the library's step per cell (work_slab128.json, %s) x %d cells" %
                    (MODE_WORK[mode], ncell),
            "kernel": "k_step<%d,false>" % {"paper": 0, "newton": 1, "mixed": 2, "mixed_seeded": 3,
                                             "newton_seeded": 4}[mode],
            "timed": "one tc_step: the three cost-ordering kernels (~2%) and the step kernel, CUDA events "
                     "on the launching stream"}


def oracle_sample(cells, head, budget_s=15.0):
    """Times the CPU oracle on growing seeded samples until about budget_s of work."""
    import oracle
    mode = 0 if head == "paper" else 1
    p = oracle.default_params(mode=mode)
    n = cells["n"].size
    rng = np.random.default_rng(99)
    m = 2048
    while True:
        idx = np.sort(rng.choice(n, min(m, n), replace=False))
        sub = synthgen.subset(cells, idx)
        a = time.perf_counter()
        oracle.step(sub, DT, p)
        el = time.perf_counter() - a
        if el * 4 > budget_s or m >= n:
            return len(idx), el, mode
        m *= 4


def cpu_baseline(cells, head):
    n, el, mode = oracle_sample(cells, head)
    cores = os.cpu_count() or 1
    return {"value": n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d seeded random cells of the same slab, oracle mode %d, OpenMP over %d threads, %.1f s"
                      % (n, mode, cores, el)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    cells = synthgen.slab(side=args.side, key=2)
    head = args.modes.split(",")[0]
    mode = 0 if head == "paper" else 1
    p = oracle.default_params(mode=mode)
    n = cells["n"].size
    per_step = 16384
    rng = np.random.default_rng(7)
    times = []
    for s in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(n, per_step, replace=False))
        sub = synthgen.subset(cells, idx)
        a = time.perf_counter()
        oracle.step(sub, DT, p)
        el = time.perf_counter() - a
        if s >= args.warmup:
            times.append(el)
    tot = float(np.sum(times))
    value = per_step * len(times) / tot
    cores = os.cpu_count() or 1
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "slab128: 128^3 TIGRESS-like slab, one step of dt = 1e4 yr", "mode": head},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d seeded random slab cells per step, oracle mode %d, %d threads" %
                                       (per_step, mode, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_configs(args):
    """Every workload config: GPU time (CUDA events, median of 3 after a warm-up; the
    48-box sweep one call after the warm-up) per mode, and the largest error against the
    oracle on sampled cells (relative on T, absolute on x_H2 and x_H+).  One JSON line."""
    import torch
    import oracle
    import paper_2210_08024_gb300 as P
    from paper_2210_08024_gb300 import tc, seed_net
    P.build()
    blob = open(seed_net.DEFAULT_BLOB, "rb").read() if os.path.exists(seed_net.DEFAULT_BLOB) else None
    stream = torch.cuda.current_stream()
    ids = {"paper": tc.TC_MODE_PAPER_FP64, "newton": tc.TC_MODE_NEWTON_FP64, "mixed": tc.TC_MODE_MIXED,
           "mixed_seeded": tc.TC_MODE_MIXED_SEEDED}

    def err(g, ref):
        return {"T_rel": float(np.max(np.abs(g["T"] - ref["T"]) / ref["T"])),
                "x_abs": float(max(np.max(np.abs(g["xH2"] - ref["xH2"])), np.max(np.abs(g["xHp"] - ref["xHp"]))))}

    def one(cells, mode, sample):
        d = tc.to_device(cells)
        pr = {k: d[k].clone() for k in STATE_KEYS}
        st = tc.Stepper(ids[mode])
        if "seeded" in mode:
            st.load_mlp(blob)
        f = tc.make_fields(d)

        def call():
            for k in STATE_KEYS:
                d[k].copy_(pr[k])
            tc.tc_step(st.h, f, DT, stream)
        ms = _time_call(call, stream, 3)
        idx = torch.from_numpy(sample).cuda()
        g = {k: d[k][idx].cpu().numpy() for k in STATE_KEYS}
        st.close()
        return ms, g

    out = {}
    rng = np.random.default_rng(17)
    work = [("1: 4096 random states", synthgen.cells_4096(), ("paper", "newton", "mixed"), None),
            ("2/4: 128^3 slab", synthgen.slab(), ("newton", "mixed", "mixed_seeded"), 3000),
            ("3: 256^3 stiff grid", synthgen.stiff(), ("mixed", "newton"), 2000)]
    for name, cells, modes, ns in work:
        n = cells["n"].size
        sample = np.arange(n) if ns is None else np.sort(rng.choice(n, ns, replace=False))
        sub = synthgen.subset(cells, sample)
        refs = {m: oracle.step(sub, DT, oracle.default_params(mode=m)) for m in ({0} if "paper" in modes else set()) | {1}}
        res = {"cells": n}
        for m in modes:
            if "seeded" in m and blob is None:
                continue
            ms, g = one(cells, m, sample)
            res[m] = {"ms": ms, "cell_updates_per_s": n / (ms * 1e-3),
                      "error_vs_oracle": err(g, refs[0 if m == "paper" else 1]),
                      "oracle_cells_compared": int(sample.size)}
        out[name] = res
        torch.cuda.empty_cache()
    # 5: 48 boxes, one batched launch replayed from a CUDA graph
    boxes = synthgen.boxes()
    res = {"boxes": len(boxes), "cells": int(sum(b[0]["n"].size for b in boxes))}
    for m in ("newton", "mixed_seeded"):
        if "seeded" in m and blob is None:
            continue
        devs = [tc.to_device(b[0]) for b in boxes]
        prs = [{k: d[k].clone() for k in STATE_KEYS} for d in devs]
        st = tc.Stepper(ids[m])
        if "seeded" in m:
            st.load_mlp(blob)
        fields = [tc.make_fields(d) for d in devs]

        def call():
            for d, pr in zip(devs, prs):
                for k in STATE_KEYS:
                    d[k].copy_(pr[k])
            tc.tc_step_batch(st.h, fields, DT, stream)
        ms = _time_call(call, stream, 1)   # ~2 min per call: one timed call after the warm-up
        worst = {"T_rel": 0.0, "x_abs": 0.0}
        for (cells, meta), d in zip(boxes, devs):
            idx = np.sort(rng.choice(cells["n"].size, 24, replace=False))
            g = {k: d[k][torch.from_numpy(idx).cuda()].cpu().numpy() for k in STATE_KEYS}
            e = err(g, oracle.step(synthgen.subset(cells, idx), DT, oracle.default_params(mode=1)))
            worst = {k: max(worst[k], e[k]) for k in worst}
        st.close()
        res[m] = {"ms": ms, "cell_updates_per_s": res["cells"] / (ms * 1e-3), "error_vs_oracle": worst,
                  "oracle_cells_compared": 24 * len(boxes), "note": "includes the state restore copies"}
        del devs, prs, fields
        torch.cuda.empty_cache()
    out["5: 48 boxes, CUDA graph"] = res
    return {"configs": out, "dt_s": DT, "data": "synthetic", "oracle": "FP64 C++ oracle on the host cores"}


def main():
    args = parse()
    if args.configs:
        print(json.dumps(run_configs(args)))
        return
    out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
