"""GPU parity of the mixed-precision mode (FP32 source terms inside the Newton
iterations, FP64 residual, update, substep length and polish) against the FP64
oracle's coupled implicit scheme: 1e-5 relative on T, 1e-6 absolute on x_H2, x_H+."""
import numpy as np
import pytest

import oracle
import synthgen
from tests._parity import assert_mixed_parity

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


@pytest.mark.parametrize("key,n", [(1, 4096), (42, 4096), (43, 4096), (78, 33), (79, 1)])
def test_mixed_random_states(tc, key, n):
    c = synthgen.cells_4096(n=n, key=key)
    ref = oracle.step(c, DT, oracle.default_params(mode=1))
    g = tc.step_numpy(c, DT, tc.TC_MODE_MIXED)
    assert np.all((g["status"] & (tc.TC_ST_NONFINITE | tc.TC_ST_MAX_SUBSTEPS)) == 0)
    assert_mixed_parity(g, ref, "mixed-key%d" % key)
    # the plain FP64 fallback is the exception, not the rule (checked on the large sample)
    if n >= 1000:
        assert np.mean((g["status"] & tc.TC_ST_FALLBACK) != 0) < 0.05


def test_mixed_slab_sampled_full_size(tc):
    import torch
    c = synthgen.slab()
    d = tc.to_device(c)
    st = tc.Stepper(tc.TC_MODE_MIXED)
    st.step(d, DT)
    torch.cuda.synchronize()
    assert tc.tc_sync_status(st.h, d["status"]) == 0
    g = tc.from_device(d)
    st.close()
    idx = np.random.default_rng(5).choice(c["n"].size, 3000, replace=False)
    ref = oracle.step(synthgen.subset(c, idx), DT, oracle.default_params(mode=1))
    assert_mixed_parity(synthgen.subset(g, idx), ref, "mixed-slab")


def test_mixed_metallicity_and_ionising_flux(tc):
    # Low and high Z' and an ionising flux exercise the grain, metal-line and
    # photoionisation terms in FP32.
    c = synthgen.cells_4096(n=512, key=91, Z=0.1)
    c["F_lyc"] = 10.0 ** np.random.default_rng(3).uniform(6.0, 10.0, 512)
    for Z in (0.1, 3.0):
        c["Zg"] = np.full(512, Z)
        c["Zd"] = np.full(512, Z)
        ref = oracle.step(c, DT, oracle.default_params(mode=1))
        g = tc.step_numpy(c, DT, tc.TC_MODE_MIXED)
        assert np.all((g["status"] & (tc.TC_ST_NONFINITE | tc.TC_ST_MAX_SUBSTEPS)) == 0)
        assert_mixed_parity(g, ref, "mixed-Z%g" % Z)
