"""Warp-cooperative step kernels (four lanes per cell) and the launch autotuner.

The cooperative kernels of the coupled FP64 Newton (mode 1) and the mixed solve (mode
2) split the four evaluations of each forward-difference Jacobian over the four lanes
of a cell.  They must reach the oracle's results at the same bars as the one-lane
kernels, on every cell (a cell that the per-cell work queue skipped or handed out
twice would show), on ragged sizes and on the hot random states that restart from the
predictor.  tc_autotune must leave the caller's state untouched, return one of its
candidate shapes, and the step in the tuned shape must still match the oracle.
"""
import numpy as np
import pytest

import oracle
import synthgen
from tests._parity import assert_fp64_parity, assert_mixed_parity

pytestmark = pytest.mark.gpu

DT = synthgen.DT_1E4YR


@pytest.fixture(scope="module")
def tc():
    import torch
    assert torch.cuda.is_available()
    import paper_2210_08024_gb300 as P
    P.build()
    from paper_2210_08024_gb300 import tc as T
    return T


def _check(tc, mode, g, ref, label):
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0), label
    if mode == tc.TC_MODE_NEWTON_FP64:
        assert_fp64_parity(g, ref, label)
        assert np.array_equal(g["nsub"], ref["nsub"]), label
    else:
        assert_mixed_parity(g, ref, label)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("key,n", [(42, 4096), (43, 4096), (80, 1), (81, 5), (82, 33), (83, 4097)])
def test_cooperative_kernel_matches_oracle(tc, mode, key, n):
    c = synthgen.cells_4096(n=n, key=key)
    ref = oracle.step(c, DT, oracle.default_params(mode=1))
    g = tc.step_numpy(c, DT, mode, lanes_per_cell=4)
    _check(tc, mode, g, ref, "coop mode%d key%d n%d" % (mode, key, n))


@pytest.mark.parametrize("mode", [1, 2])
def test_cooperative_and_one_lane_kernels_agree_on_slab_sample(tc, mode):
    c = synthgen.slab(ncell=20000, key=14)
    a = tc.step_numpy(c, DT, mode, lanes_per_cell=1)
    b = tc.step_numpy(c, DT, mode, lanes_per_cell=4)
    if mode == 1:
        assert_fp64_parity(b, a, "coop vs one lane")
        assert np.array_equal(a["nsub"], b["nsub"])
    else:
        assert_mixed_parity(b, a, "coop vs one lane (mixed)")


@pytest.mark.parametrize("mode", [1, 2])
def test_autotune_keeps_state_and_tuned_step_matches_oracle(tc, mode):
    import torch
    c = synthgen.cells_4096(n=3000, key=84)
    d = tc.to_device(c)
    before = {k: d[k].clone() for k in ("T", "xH2", "xHp")}
    st = tc.Stepper(mode)
    choice = st.autotune(d, DT)
    torch.cuda.synchronize()
    for k, v in before.items():
        assert torch.equal(d[k], v), k
    assert choice["block"] in (32, 64, 128)
    assert choice["blocks_per_sm"] in (0, 4)
    assert choice["lanes_per_cell"] in (1, 4)
    assert choice["ms"] > 0.0
    st.step(d, DT)
    torch.cuda.synchronize()
    g = tc.from_device(d)
    st.close()
    ref = oracle.step(c, DT, oracle.default_params(mode=1))
    _check(tc, mode, g, ref, "autotuned mode%d" % mode)


def test_autotune_rejects_bad_arguments(tc):
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64)
    f = tc.tc_fields()
    f.ncell = 0
    c = tc.tc_tune_choice()
    import ctypes
    assert tc.lib.tc_autotune(st.h, ctypes.byref(f), DT, None, ctypes.byref(c)) == tc.TC_EINVAL
    st.close()
