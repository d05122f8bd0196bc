"""Launch-shape autotuner of the step kernel.

The step kernel is persistent: its grid is SMs x resident blocks, and each lane takes
cells from a work queue until it is empty.  Two knobs shape it: the block size
(tc_params.block: 32..128 threads, the kernels are compiled for at most 128) and the
number of blocks per SM (tc_params.blocks_per_sm; 0 lets the occupancy calculator
decide).  Per-lane register use is high (up to 255 registers), so fewer, smaller
blocks can trade occupancy for instruction-cache and scheduling behaviour.  This
module times every candidate on a sample of the workload with CUDA events (median of
`reps` launches after one warm-up) and picks the fastest.  Results are cached in a
JSON file keyed by GPU name, mode and workload name.
"""
from __future__ import annotations

import json
import os

from . import tc

CANDIDATES = [(b, k) for b in (32, 64, 96, 128) for k in (0, 1, 2, 4, 8)]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "tc_gb300_autotune.json")


def _time_launch(mode: int, dev: dict, dt: float, block: int, bps: int, reps: int, blob=None) -> float:
    import torch
    st = tc.Stepper(mode, block=block, blocks_per_sm=bps)
    if blob is not None:
        st.load_mlp(blob)
    pristine = {k: dev[k].clone() for k in ("T", "xH2", "xHp")}
    f = tc.make_fields(dev)
    times = []
    stream = torch.cuda.current_stream()
    for r in range(reps + 1):
        for k, v in pristine.items():
            dev[k].copy_(v)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tc.tc_step(st.h, f, dt, stream)
        e1.record(stream)
        e1.synchronize()
        if r > 0:
            times.append(e0.elapsed_time(e1))
    for k, v in pristine.items():
        dev[k].copy_(v)
    st.close()
    times.sort()
    return times[len(times) // 2]


def tune(mode: int, dev: dict, dt: float, workload: str, reps: int = 3, blob=None, cache: str | None = DEFAULT_CACHE,
         candidates=CANDIDATES, log=None) -> dict:
    """Returns {"block", "blocks_per_sm", "ms", "table"} for `mode` on the device sample
    `dev` (a dict of device tensors as made by tc.to_device).  Uses the cache when it
    holds an entry for this GPU, mode and workload."""
    import torch
    key = "%s|mode%d|%s" % (torch.cuda.get_device_name(), mode, workload)
    db = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as fh:
                db = json.load(fh)
        except (OSError, ValueError):
            db = {}
    if key in db:
        return db[key]
    table = []
    for block, bps in candidates:
        ms = _time_launch(mode, dev, dt, block, bps, reps, blob)
        table.append((block, bps, ms))
        if log:
            log("  block %3d blocks/SM %d: %.2f ms" % (block, bps, ms))
    block, bps, ms = min(table, key=lambda t: t[2])
    res = {"block": block, "blocks_per_sm": bps, "ms": ms, "table": table}
    if cache:
        db[key] = res
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            with open(cache, "w") as fh:
                json.dump(db, fh, indent=1)
        except OSError:
            pass
    return res
