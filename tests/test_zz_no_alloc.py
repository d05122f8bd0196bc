"""tc_step_host_static: the host-buffer step for callers that may not allocate device
memory (no handle, no cudaMalloc; device staging in the library's static scratch).

Its results must match the handle-based host entry point tc_step_host at the FP64
parity tolerance, on two calls in a row.  The second call is smaller and uses other
inputs, so anything stale that the first call left in the shared scratch, such as the
work-queue cursor, would show.  Every mode it accepts (the paper's scheme, the coupled
FP64 Newton and the mixed solve) is also checked against the CPU oracle.  The file is
named to be collected last."""
import numpy as np
import pytest

import oracle
import synthgen
from tests._parity import assert_fp64_parity, assert_mixed_parity, ulp_spread

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


def _host_arrays(tc, cells):
    n = cells["n"].size
    h = {k: np.ascontiguousarray(np.broadcast_to(np.asarray(cells[k], dtype=np.float64), (n,))).copy()
         for k in tc.INPUT_KEYS + ("T", "xH2", "xHp")}
    for k in ("xe", "xCp", "xCO"):
        h[k] = np.zeros(n)
    h["nsub"] = np.zeros(n, dtype=np.int32)
    h["status"] = np.zeros(n, dtype=np.int32)
    return h


def test_static_entry_matches_host_entry_twice(tc):
    params = tc.tc_params_default(tc.TC_MODE_NEWTON_FP64)
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64)
    for n, key in ((3000, 501), (1500, 502)):
        cells = synthgen.cells_4096(n=n, key=key)
        a = _host_arrays(tc, cells)
        b = _host_arrays(tc, cells)
        tc.tc_step_host_static(params, tc.make_host_fields(a), DT)
        st.step_host(b, DT)
        assert_fp64_parity(a, b, "static-vs-host n=%d" % n)
        for k in ("xe", "xCp", "xCO"):
            np.testing.assert_allclose(a[k], b[k], rtol=1e-9, atol=1e-14)
        # error bits equal; the informational ones (predictor restart and the like)
        # belong to the solver's path, which differs between the one-lane kernel
        # (one iteration per trip) and the four-lane one tc_step_host picks here
        assert np.array_equal(a["nsub"], b["nsub"])
        assert np.array_equal(a["status"] & tc.TC_ST_ERROR_MASK, b["status"] & tc.TC_ST_ERROR_MASK)
    st.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_static_entry_matches_oracle_in_every_mode(tc, mode):
    params = tc.tc_params_default(mode)
    for n, key in ((2000, 511), (700, 512)):
        cells = synthgen.cells_4096(n=n, key=key)
        a = _host_arrays(tc, cells)
        tc.tc_step_host_static(params, tc.make_host_fields(a), DT)
        if mode == 0:
            ref, spread = ulp_spread(oracle, cells, DT, oracle.default_params(mode=0))
            assert_fp64_parity(a, ref, "static mode0 n=%d" % n, spread=spread)
        else:
            ref = oracle.step(cells, DT, oracle.default_params(mode=1))
            assert np.all((a["status"] & tc.TC_ST_ERROR_MASK) == 0)
            if mode == 1:
                assert_fp64_parity(a, ref, "static mode1 n=%d" % n)
                assert np.array_equal(a["nsub"], ref["nsub"])
            else:
                assert_mixed_parity(a, ref, "static mixed n=%d" % n)


def test_static_entry_rejects_more_cells_than_its_scratch(tc):
    params = tc.tc_params_default(tc.TC_MODE_NEWTON_FP64)
    f = tc.tc_fields()
    f.ncell = tc.TC_STATIC_MAX_CELLS + 1
    assert tc.lib.tc_step_host_static(params, f, DT, None) == tc.TC_EINVAL
    with pytest.raises(ValueError):
        tc.tc_step_host_static(params, f, DT)
