"""Host-side arithmetic of the benchmark line, without a GPU: the FP64 work weighting,
the roofline entry and the work counts it reads."""
import pytest

import bench


def test_flops_weighting():
    counts = {"add": 10.0, "mul": 20.0, "div": 1.0, "sqrt": 2.0, "exp": 3.0, "log": 4.0}
    w = {"div": 5.0, "sqrt": 8.0, "exp": 16.0, "log": 30.0}
    # adds and multiplies count 1 each; every other class its FMA slots at 2 flops per slot
    assert bench.flops_per_cell(counts, w) == pytest.approx(30.0 + 2.0 * (5.0 + 16.0 + 48.0 + 120.0))


def test_roofline_entry():
    work = bench.work_per_cell()
    peaks = {"fp64_fma_per_s": 5e11, "weights": {"div": 5.7, "sqrt": 8.6, "exp": 16.0, "log": 30.2}}
    r = {"kernel_ms": 400.0}
    ncell = 2097152
    rl = bench.roofline_of(work, r, "newton", ncell, peaks)
    fl = bench.flops_per_cell(work["mode1"], peaks["weights"]) * ncell
    assert rl["achieved"] == pytest.approx(fl / 0.4 / 1e12)
    assert rl["peak"] == pytest.approx(1.0)
    assert rl["frac"] == pytest.approx(rl["achieved"] / rl["peak"])
    if bench.TRAFFIC_BYTES_PER_CELL:
        assert rl["traffic"] == pytest.approx(bench.TRAFFIC_BYTES_PER_CELL * ncell)
    else:  # no capture of the current kernel: no traffic figure
        assert rl["traffic"] is None
    assert bench.roofline_of(work, r, "mixed", ncell, peaks)["traffic"] is None


def test_work_counts_cover_every_mode():
    work = bench.work_per_cell()
    for m in ("mode0", "mode1"):
        assert all(work[m][k] > 0 for k in ("add", "mul", "div", "exp", "log"))
    # the coupled implicit scheme does more FP64 work per cell than the sequential one
    assert work["mode1"]["exp"] > work["mode0"]["exp"]
    # the mixed path evaluates its physics in FP32 and df64 only: its FP64 work is the
    # Newton update, the residuals and the closure
    assert work["mode2"]["exp"] == 0 and work["mode2"]["log"] == 0 and work["mode2"]["add"] > 0
    assert all(work["mode2_df64"][k] > 0 for k in ("add", "mul", "div", "exp", "log"))
    assert all(work["mode2_fp32"][k] > 0 for k in ("add", "mul", "div", "exp", "log"))


def test_work_breakdown_covers_the_counted_work():
    import json
    from paper_2210_08024_gb300 import work
    with open(work.OUT) as fh:
        res = json.load(fh)
    rows = work.breakdown(res, "mode1")
    names = [r[0] for r in rows]
    # the FP64 Newton step's blocks, the stepped temperature column among them
    for blk in ("source", "chem_T", "cool_T", "temp_step", "equil_it", "newton64_it"):
        assert blk in names
    # largest first, and the blocks add up to the weighted per-cell count
    assert all(rows[i][2] >= rows[i + 1][2] for i in range(len(rows) - 1))
    per_cell = res["per_cell"]["mode1"]
    total = sum(per_cell[c] * work.SLOT_WEIGHTS[c] for c in work.CLASSES)
    assert sum(r[2] for r in rows) == pytest.approx(total, rel=1e-3)
