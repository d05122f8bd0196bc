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
