"""GPU parity of the PDR slab driver (tc_pdr, Secs. 7.2, 7.3) against the oracle's
driver (oracle/pdr.py), and the transition columns of a Fig. f:HIH2-noCR-like suite
against the analytic approximation the paper prints (Eq. e:NH_trans)."""
import numpy as np
import pytest

import oracle
from oracle import pdr
from tests._parity import assert_fp64_parity, assert_mixed_parity

pytestmark = pytest.mark.gpu

MYR = 1e6 * oracle.YEAR_S


@pytest.fixture(scope="module")
def tc():
    import torch
    assert torch.cuda.is_available()
    import paper_2210_08024_gb300 as P
    P.build()
    from paper_2210_08024_gb300 import tc as T
    return T


def _slabs():
    n = np.array([1e2, 1e3, 1e2, 30.0])
    chi0 = np.array([1.0, 1e2, 1.0, 10.0])
    xi0 = np.array([0.0, 0.0, 2e-16, 2e-16])
    Z = np.array([1.0, 1.0, 1.0, 0.5])
    dx = pdr.bialy_sternberg_ntrans(chi0, n) / 25.0 / n
    return n, chi0, xi0, Z, dx


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _flat(d):
    return {k: d[k].ravel() for k in ("T", "xH2", "xHp")}


@pytest.mark.parametrize("mode", [1, 2])
def test_slabs_match_oracle(tc, mode):
    import torch
    n, chi0, xi0, Z, dx = _slabs()
    ncell, tend, nchunk = 100, 120.0, 120
    ref = pdr.slabs(n, chi0, xi0, Z, dx, ncell, oracle.default_params(mode=1, flags=oracle.F_CONST_KGR),
                    t_end=tend * MYR, nchunk=nchunk)
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64 if mode == 1 else tc.TC_MODE_MIXED, flags=tc.TC_CONST_KGR)
    g = _host(st.pdr(n, chi0, xi0, Z, dx, ncell, t_end_s=tend * MYR, nchunk=nchunk))
    torch.cuda.synchronize()
    st.close()
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0)
    if mode == 1:
        assert np.array_equal(g["status"], ref["status"])
        assert_fp64_parity(_flat(g), _flat(ref), "pdr")
        np.testing.assert_allclose(g["N_trans"], ref["N_trans"], rtol=1e-8)
        np.testing.assert_allclose(g["N_c"], ref["N_c"], rtol=1e-13)
        np.testing.assert_allclose(g["chi_pe"], ref["chi_pe"], rtol=1e-9, atol=1e-300)
        np.testing.assert_allclose(g["f_h2"], ref["f_h2"], rtol=1e-9)
    else:
        assert_mixed_parity(_flat(g), _flat(ref), "pdr mixed")
        np.testing.assert_allclose(g["N_trans"], ref["N_trans"], rtol=1e-3)


def suite():
    """Sec. 7.3 suite without CRs: n = 10..1e4 x chi0 = 0.1..1e4, keeping the points the
    paper could resolve (N_trans over more than three cells of at least 1e-3 pc)."""
    nn, cc = np.meshgrid([10.0, 1e2, 1e3, 1e4], [0.1, 1.0, 10.0, 1e2, 1e3, 1e4])
    n, chi0 = nn.ravel(), cc.ravel()
    Nt = pdr.bialy_sternberg_ntrans(chi0, n)
    keep = Nt / n >= 3 * 1e-3 * 3.0856775814913673e18
    return n[keep], chi0[keep], Nt[keep]


def test_transition_suite_against_analytic_approximation(tc):
    # The transition column resolved by ~25 cells, the slab 4 times deeper; each within a
    # factor 1.5 of Eq. e:NH_trans.  (Without CRs, cells far behind the transition of
    # strongly lit slabs cool to ~2 K and need thousands of substeps per chunk; N_trans
    # does not depend on them.)
    import torch
    n, chi0, Nt = suite()
    assert n.size == 19
    dx = Nt / 25.0 / n
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64, flags=tc.TC_CONST_KGR)
    g = _host(st.pdr(n, chi0, np.zeros_like(n), np.ones_like(n), dx, 100, t_end_s=300 * MYR, nchunk=300))
    torch.cuda.synchronize()
    st.close()
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0)
    ratio = g["N_trans"] / Nt
    assert np.all((ratio > 1 / 1.5) & (ratio < 1.5)), ratio


def test_invalid_specs_rejected(tc):
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64)
    with pytest.raises(tc.TcError):
        st.pdr([1e2], [1.0], [0.0], [1.0], [0.0], 10)
    with pytest.raises(tc.TcError):
        st.pdr([1e2], [1.0], [0.0], [1.0], [1e17], 0)
    st.close()
