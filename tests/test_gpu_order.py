"""The cost-ordered work queue (tc_params.order_cells): cells are handed to the
persistent kernel in decreasing order of their predicted substep count, and every
result is bit-for-bit the one of index order (each cell's arithmetic does not depend
on the lane or the time it runs).  A cell skipped or processed twice would differ."""
import numpy as np
import pytest

import synthgen

pytestmark = pytest.mark.gpu

DT = synthgen.DT_1E4YR
KEYS = ("T", "xH2", "xHp", "xe", "xCO", "nsub", "status", "iters")


@pytest.fixture(scope="module")
def tc():
    import torch
    assert torch.cuda.is_available()
    import paper_2210_08024_gb300 as P
    P.build()
    from paper_2210_08024_gb300 import tc as T
    return T


def _run(tc, cells, mode, order):
    import torch
    d = tc.to_device(cells)
    st = tc.Stepper(mode, order_cells=order)
    st.step(d, DT)
    torch.cuda.synchronize()
    st.close()
    return tc.from_device(d)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("workload", ["random", "slab", "ragged"])
def test_order_does_not_change_results(tc, mode, workload):
    c = {"random": lambda: synthgen.cells_4096(n=4096, key=9),
         "slab": lambda: synthgen.slab(ncell=50000, key=10),
         "ragged": lambda: synthgen.cells_4096(n=257, key=11)}[workload]()
    a = _run(tc, c, mode, 0)
    b = _run(tc, c, mode, 1)
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


def test_order_in_batched_graph(tc):
    import torch
    boxes = [synthgen.cells_4096(n=n, key=20 + i) for i, n in enumerate((1000, 3000, 513))]
    outs = {}
    for order in (0, 1):
        devs = [tc.to_device(b) for b in boxes]
        st = tc.Stepper(tc.TC_MODE_NEWTON_FP64, order_cells=order)
        tc.tc_step_batch(st.h, [tc.make_fields(d) for d in devs], DT)
        torch.cuda.synchronize()
        st.close()
        outs[order] = [tc.from_device(d) for d in devs]
    for a, b in zip(outs[0], outs[1]):
        for k in KEYS:
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("mode", [1, 2])
def test_cost_hint_does_not_change_results(tc, mode):
    # a second step ordered by the first step's Newton iterations, and one ordered by a
    # meaningless hint, give the results of index order bit for bit
    import torch
    c = synthgen.slab(ncell=50000, key=12)
    d = tc.to_device(c)
    st = tc.Stepper(mode)
    st.step(d, DT)
    torch.cuda.synchronize()
    start = {k: d[k].clone() for k in ("T", "xH2", "xHp")}
    hints = {"previous": d["iters"].clone(),
             "random": torch.randint(0, 1000, (c["n"].size,), dtype=torch.int32, device="cuda")}
    outs = {}
    for name in ("none", "previous", "random"):
        for k in start:
            d[k].copy_(start[k])
        d["cost_hint"] = hints.get(name)
        s2 = tc.Stepper(mode, order_cells=0 if name == "none" else 1)
        s2.step(d, DT)
        torch.cuda.synchronize()
        s2.close()
        outs[name] = tc.from_device(d)
    st.close()
    for name in ("previous", "random"):
        for k in KEYS:
            assert np.array_equal(outs["none"][k], outs[name][k]), (name, k)
