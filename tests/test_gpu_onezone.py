"""GPU parity of the one-zone equilibrium-curve driver (tc_eq_curves, Sec. 7.1)
against the oracle's driver (oracle/onezone.py): the settled states element by element,
the pressures, and the curves' extrema indices."""
import numpy as np
import pytest

import oracle
from oracle import onezone as oz
from tests._parity import RTOL_FP64, assert_fp64_parity, assert_mixed_parity

pytestmark = pytest.mark.gpu

MYR = oz.MYR_S


@pytest.fixture(scope="module")
def tc():
    import torch
    assert torch.cuda.is_available()
    import paper_2210_08024_gb300 as P
    P.build()
    from paper_2210_08024_gb300 import tc as T
    return T


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _flat(d):
    return {k: d[k].ravel() for k in ("T", "xH2", "xHp")}


def _check_extrema(g, ref, rtol):
    # The index is unique unless two neighbouring pressures tie within the tolerance;
    # then either neighbour is a valid answer.
    for c in range(ref["P"].shape[0]):
        for key in ("i_max", "i_min"):
            a, b = int(g[key][c]), int(ref[key][c])
            if a == b:
                continue
            P = ref["P"][c]
            lo = min(a, b)
            assert abs(a - b) == 1 and lo >= 0 and abs(P[lo + 1] - P[lo]) <= 4 * rtol * abs(P[lo]), (key, c, a, b)


def _unsh_args():
    chi0 = np.array([1.0, 10.0, 1.0, 1.0])
    Zg = np.array([1.0, 1.0, 0.1, 0.1])
    Zd = np.array([1.0, 1.0, 0.1, 0.025])
    return chi0, 2e-16 * chi0, Zg, Zd


@pytest.mark.parametrize("mode", [1, 0])
def test_unshielded_curves_fp64(tc, mode):
    import torch
    n = np.logspace(-1, 4, 61)
    chi0, xi0, Zg, Zd = _unsh_args()
    ref = oz.curves(n, chi0, xi0, Zg, Zd, oracle.default_params(mode=mode, flags=oracle.F_CONST_KGR),
                    t_end=1e2 * MYR, nchunk=10)
    mode_id = tc.TC_MODE_NEWTON_FP64 if mode == 1 else tc.TC_MODE_PAPER_FP64
    st = tc.Stepper(mode_id, flags=tc.TC_CONST_KGR)
    g = _host(st.eq_curves(n, chi0, xi0, Zg, Zd, t_end_s=1e2 * MYR, nchunk=10))
    torch.cuda.synchronize()
    st.close()
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0)
    assert np.array_equal(g["status"], ref["status"])
    assert_fp64_parity(_flat(g), _flat(ref), "unshielded mode %d" % mode)
    np.testing.assert_allclose(g["P"], ref["P"], rtol=RTOL_FP64, atol=0)
    np.testing.assert_allclose(g["xe"], ref["xe"], rtol=RTOL_FP64, atol=1e-14)
    _check_extrema(g, ref, RTOL_FP64)
    assert np.all(g["i_max"] >= 0) and np.all(g["i_min"] > g["i_max"])


def test_shielded_curves_fp64(tc):
    import torch
    n = np.logspace(-1, 6, 36)
    chi0 = np.array([1.0, 10.0])
    xi0 = np.array([2e-16, 2e-16])
    Z = np.array([1.0, 1.0])
    p = oracle.default_params(mode=1, flags=oracle.F_CONST_KGR, T_cmb=6.0, tau_opt_over_tau_pe=1 / 1.87)
    ref = oz.curves(n, chi0, xi0, Z, Z, p, t_end=1e2 * MYR, nchunk=50, shielded=True)
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64, flags=tc.TC_CONST_KGR, T_cmb=6.0, tau_opt_over_tau_pe=1 / 1.87)
    g = _host(st.eq_curves(n, chi0, xi0, Z, Z, shielded=True, t_end_s=1e2 * MYR, nchunk=50))
    torch.cuda.synchronize()
    st.close()
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0)
    assert_fp64_parity(_flat(g), _flat(ref), "shielded")
    np.testing.assert_allclose(g["xCO"], ref["xCO"], rtol=RTOL_FP64, atol=1e-16)
    np.testing.assert_allclose(g["chg"], ref["chg"], rtol=1e-3, atol=1e-12)
    _check_extrema(g, ref, RTOL_FP64)


def test_unshielded_curves_mixed(tc):
    import torch
    n = np.logspace(-1, 4, 61)
    chi0, xi0, Zg, Zd = _unsh_args()
    ref = oz.curves(n, chi0, xi0, Zg, Zd, oracle.default_params(mode=1, flags=oracle.F_CONST_KGR),
                    t_end=1e2 * MYR, nchunk=10)
    st = tc.Stepper(tc.TC_MODE_MIXED, flags=tc.TC_CONST_KGR)
    g = _host(st.eq_curves(n, chi0, xi0, Zg, Zd, t_end_s=1e2 * MYR, nchunk=10))
    torch.cuda.synchronize()
    st.close()
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0)
    assert_mixed_parity(_flat(g), _flat(ref), "unshielded mixed")
    assert np.all(np.abs(g["i_max"] - ref["i_max"]) <= 1) and np.all(np.abs(g["i_min"] - ref["i_min"]) <= 1)


def test_single_density_and_repeat_calls(tc):
    # nn = 1 (no extrema) and a second call on the same handle with a larger grid
    import torch
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64, flags=tc.TC_CONST_KGR)
    g1 = _host(st.eq_curves([30.0], [1.0], [2e-16], [1.0], [1.0], t_end_s=1e2 * MYR, nchunk=3))
    g2 = _host(st.eq_curves(np.logspace(0, 2, 70), np.ones(3), 2e-16 * np.ones(3), np.ones(3), np.ones(3),
                            t_end_s=1e2 * MYR, nchunk=3))
    torch.cuda.synchronize()
    st.close()
    assert g1["i_max"][0] == -1 and g1["i_min"][0] == -1
    r1 = oz.curves([30.0], [1.0], [2e-16], [1.0], [1.0], oracle.default_params(mode=1, flags=oracle.F_CONST_KGR),
                   t_end=1e2 * MYR, nchunk=3)
    assert g1["T"][0, 0] == pytest.approx(r1["T"][0, 0], rel=RTOL_FP64)
    # three identical curves give identical rows
    assert np.array_equal(g2["T"][0], g2["T"][1]) and np.array_equal(g2["T"][0], g2["T"][2])


def test_invalid_specs_rejected(tc):
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64)
    with pytest.raises(tc.TcError):
        st.eq_curves([1.0, -1.0], [1.0], [2e-16], [1.0], [1.0])
    with pytest.raises(tc.TcError):
        st.eq_curves([1.0], [1.0], [2e-16], [1.0], [1.0], nchunk=0)
    with pytest.raises(tc.TcError):
        st.eq_curves([1.0], [1.0], [2e-16], [1.0], [1.0], xH2_init=0.4, xHp_init=0.5)
    st.close()
