"""Pins of the oracle's PDR slab driver (Secs. 7.2, 7.3): the HI-to-H2 transition column
against the analytic approximation the paper prints (Eqs. e:alpha, e:G, e:NH_trans),
its dependence on chi0/n only, the steady state, photon bookkeeping of the beamed field,
and the transition-column interpolation."""
import numpy as np
import pytest

import oracle
from oracle import pdr

MYR = 1e6 * oracle.YEAR_S


def _run(n, chi0, cells_per_ntrans=30.0, ncell=400, t_end=200.0, nchunk=200, xi0=0.0):
    Nt = pdr.bialy_sternberg_ntrans(chi0, n)
    dx = Nt / cells_per_ntrans / n
    p = oracle.default_params(mode=1, flags=oracle.F_CONST_KGR)
    return Nt, pdr.slabs([n], [chi0], [xi0], [1.0], [dx], ncell, p, t_end=t_end * MYR, nchunk=nchunk)


@pytest.mark.parametrize("n,chi0", [(1e2, 1.0), (1e3, 1e2), (10.0, 1.0), (1e4, 1.0)])
def test_transition_column_matches_analytic_approximation(n, chi0):
    # Sec. 7.3, no CRs and constant k_gr: the numerical transition column follows the
    # Bialy & Sternberg approximation (agreement "quite well" in Fig. f:HIH2-noCR).
    Nt, r = _run(n, chi0)
    assert np.all(r["status"] == 0)
    assert 1 / 1.5 < r["N_trans"][0] / Nt < 1.5


def test_transition_depends_on_chi0_over_n_only():
    # alpha G is proportional to chi0 / n (Sec. 7.3): scaling both by 10 leaves N_trans.
    _, a = _run(1e2, 1.0)
    _, b = _run(1e3, 10.0)
    assert b["N_trans"][0] == pytest.approx(a["N_trans"][0], rel=0.02)


def test_strong_field_transition_is_sharp_and_weak_field_gradual():
    # Strong field (alpha G >> 1): H2 rises from 10% to 90% of 0.5 within a narrow
    # column range; weak field (alpha G << 1): the rise is gradual (Sec. 7.3).
    def width(r):
        y = 2 * r["xH2"][0]
        N = r["N_c"][0]
        return N[np.argmax(y >= 0.9)] / N[np.argmax(y >= 0.1)]
    _, strong = _run(10.0, 30.0)
    _, weak = _run(1e4, 1.0, ncell=600)
    assert width(strong) < 2.0
    assert width(weak) > 2.0 * width(strong)


def test_steady_state_reached():
    Nt, r1 = _run(1e2, 1.0, t_end=200.0, nchunk=200)
    _, r2 = _run(1e2, 1.0, t_end=400.0, nchunk=400)
    assert r2["N_trans"][0] == pytest.approx(r1["N_trans"][0], rel=1e-3)
    np.testing.assert_allclose(r2["xH2"][0], r1["xH2"][0], atol=1e-4)


def test_beamed_field_photon_bookkeeping():
    # The cell-averaged fields times the cells' optical depths add up to the photons
    # absorbed by the whole slab: sum_k dtau_k chi_k / chi0 = 1 - exp(-tau_total).
    rng = np.random.default_rng(3)
    n = rng.lognormal(3.0, 1.0, 300)
    dx = 1e17
    chi_pe, chi_lw, f_h2, xi, N_c = pdr.beamed_fields(n, np.zeros_like(n), dx, 2.0, 2e-16, 1.0)
    for chi, sig in ((chi_pe, pdr.SIGMA_PE), (chi_lw, pdr.SIGMA_LW)):
        dtau = sig * n * dx
        assert np.sum(dtau * chi / 2.0) == pytest.approx(1.0 - np.exp(-dtau.sum()), rel=1e-12)
    assert np.all(np.diff(N_c) > 0) and N_c[0] == pytest.approx(0.5 * n[0] * dx)


def test_transition_column_interpolation():
    N = np.array([1.0, 3.0, 5.0, 7.0])
    assert pdr.transition_column(N, np.array([0.0, 0.1, 0.3, 0.5])) == pytest.approx(3.0 + 2.0 * (0.5 - 0.2) / 0.4)
    assert pdr.transition_column(N, np.array([0.3, 0.4, 0.5, 0.5])) == 1.0
    assert pdr.transition_column(N, np.zeros(4)) == -1.0
