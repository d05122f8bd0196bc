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
# DRAM bytes per cell of one k_step<1> launch, from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum on a 112^3 slab, profiles/k_step_fp64_slab128.md), scaled by cells.
TRAFFIC_BYTES_PER_CELL = 138.9


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
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def work_per_cell():
    """FP64 operations per cell by class (add, mul, div, sqrt, exp, log) of one step on
    the slab, per mode, counted from the library's own step functions
    (paper_2210_08024_gb300/work.py)."""
    path = os.path.join(ROOT, "paper_2210_08024_gb300", "work_slab128.json")
    with open(path) as fh:
        return json.load(fh)["per_cell"]


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
                           ("fma32", 1, iters * 8)):
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
    return {"fp64_fma_per_s": fma, "fp32_fma_per_s": rates["fma32"], "rates": rates, "weights": weights}


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

    cells = synthgen.slab(side=args.side, key=2 + rank)
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
        if ws > 1:
            import torch.distributed as dist
            tt = torch.tensor([ms], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms = float(tt.item())
        nbad = tc.tc_sync_status(st.h, dev["status"])
        results[mname] = {"ms_per_step": ms / args.steps, "kernel_ms": float(np.mean(kms)),
                          "value": ws * ncell * args.steps / (ms * 1e-3), "launches": launches,
                          "cells_not_ok": nbad, "newton_iters_per_cell": float(dev["iters"].double().mean().item()),
                          "mode_id": mode_ids[mname]}
        st.close()

    head = modes[0]
    e2e = None if args.no_e2e else run_e2e(args, tc, torch, cells, ncell, mode_ids[head], stream, barrier, ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return None
    return report(args, results, head, ncell, peaks, e2e, clocks, cells, ws)


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
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([e2e_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    st.close()
    return {"value": ws * ncell * args.steps / (e2e_ms * 1e-3), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "api": "tc_step_host"}


def report(args, results, head, ncell, peaks, e2e, clocks, cells, ws):
    # roofline of the step kernel (FP64 pipe): the FP64 work of one launch (per-cell
    # counts of the library's own step, weighted by the FMA-slot cost of each operation
    # class measured in this run) over the CUDA-event duration of the launch.
    work = work_per_cell()
    r = results[head]
    roofline = None
    if peaks is not None:
        roofline = roofline_of(work, r, head, ncell, peaks)
        for name, rr in results.items():
            rl = roofline_of(work, rr, name, ncell, peaks)
            rr["fp64_roofline_frac"] = rl["frac"]
            rr["fp64_tflops"] = rl["achieved"]
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
               "fma_slot_weights": peaks["weights"]},
           "cpu_baseline": cpu}
    return out


def roofline_of(work, r, mode, ncell, peaks):
    fl = flops_per_cell(work[MODE_WORK[mode]], peaks["weights"]) * ncell
    achieved = fl / (r["kernel_ms"] * 1e-3) / 1e12
    peak = 2.0 * peaks["fp64_fma_per_s"] / 1e12
    return {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": TRAFFIC_BYTES_PER_CELL * ncell if mode == "newton" else None,
            "peak_source": "measured FP64 FMA rate (library microbenchmark, this run); nominal %.2f" %
                           FP64_NOMINAL_TFLOPS,
            "work": "FP64 flops of the library's step per cell (work_slab128.json, %s) x %d cells" %
                    (MODE_WORK[mode], ncell),
            "kernel": "k_step<%d,false>" % {"paper": 0, "newton": 1, "mixed": 2, "mixed_seeded": 3,
                                             "newton_seeded": 4}[mode]}


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


def main():
    args = parse()
    out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
