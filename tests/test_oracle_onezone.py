"""Pins of the oracle's one-zone equilibrium-curve driver (Sec. 7.1) and of the
shielding prescriptions it uses (Eqs. e:fshld_H2_DB, e:cratt; Sec. 7.1.2): statements
and numbers the paper prints, and the steady state that the settled cells must satisfy."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import onezone as oz

HERE = os.path.dirname(os.path.abspath(__file__))
A = json.load(open(os.path.join(HERE, "golden", "paper_anchors.json")))


# ------------------------------------------------------------------ shielding pieces
def test_h2_self_shielding_shape():
    a = A["fshld_h2_shape"]
    # optically thin line cores below ~1e14, thick above
    assert oz.f_shld_h2(1e12) > 0.98
    assert oz.f_shld_h2(a["core_thick_N"] * 10) < 0.5
    # Lorentzian-wing regime: local log-slope near -1/2 over the lower part of 1e17..5e20
    # (the printed form steepens towards 5e20, where line overlap sets in)
    for N in np.logspace(np.log10(a["wing_N_range"][0]) + 0.5, 19.0, 5):
        s = (np.log(oz.f_shld_h2(N * 1.01)) - np.log(oz.f_shld_h2(N / 1.01))) / (2 * np.log(1.01))
        assert s == pytest.approx(a["wing_slope"], abs=0.08), N
    # the Doppler parameter no longer matters once the wings dominate
    N = 10 * a["b5_insensitive_N"]
    assert oz.f_shld_h2(N, b5=1.0) == pytest.approx(oz.f_shld_h2(N, b5=3.0), rel=0.02)
    assert oz.f_shld_h2(1e14, b5=1.0) < 0.8 * oz.f_shld_h2(1e14, b5=3.0)


def test_cr_attenuation_onset_and_slope():
    a = A["cr_attenuation_onset"]
    N_onset = a["A_V"] * a["NH_per_AV"]
    assert N_onset == pytest.approx(oz.N0_CR, rel=0.01)
    assert oz.xi_attenuated(2e-16, 0.9 * N_onset) == 2e-16
    # xi ~ A_V^-1 beyond the onset
    for av in (1.0, 5.0, 50.0):
        assert oz.xi_attenuated(2e-16, av * a["NH_per_AV"]) == pytest.approx(2e-16 * a["A_V"] / av, rel=0.01)


def test_shielding_length_anchor():
    a = A["shielded_equilibrium"]
    n = 10 ** a["log10_n_cr_over_pe"]
    N = n * oz.shielding_length_cm(n)
    assert N == pytest.approx(a["N_shld_at_cr_over_pe"], rel=0.01)


def test_extrema_rule():
    P = np.array([1.0, 2.0, 3.0, 2.5, 2.0, 2.2, 5.0])
    assert oz.extrema(P) == (2, 4)
    assert oz.extrema(np.arange(5.0)) == (-1, -1)
    assert oz.extrema(np.array([3.0, 2.0, 1.0])) == (0, -1)
    assert oz.extrema(np.array([1.0, 1.0, 0.5, 0.5, 0.7])) == (1, 3)


# ------------------------------------------------------------------ unshielded curves
def _unshielded(chi0=(1.0,), Z=(1.0,), n=None):
    n = np.logspace(-1, 3.5, 91) if n is None else n
    chi0 = np.asarray(chi0, dtype=float)
    Z = np.asarray(Z, dtype=float)
    p = oracle.default_params(mode=1, flags=oracle.F_CONST_KGR)
    return n, oz.curves(n, chi0, 2e-16 * chi0, Z, Z, p, nchunk=10)


def test_unshielded_curve_matches_printed_extrema():
    a = A["unshielded_equilibrium"]
    n, r = _unshielded()
    assert np.all(r["status"] == 0)
    imax, imin = r["i_max"][0], r["i_min"][0]
    assert 0 <= imax < imin
    P = r["P"][0]
    assert a["Pmax_k"] / 2 < P[imax] < a["Pmax_k"] * 2
    assert a["Pmin_k"] / 2 < P[imin] < a["Pmin_k"] * 2
    assert a["n_max"] / 2 < n[imax] < a["n_max"] * 2
    assert a["n_min"] / 2.5 < n[imin] < a["n_min"] * 2
    assert a["T_max"] / 1.5 < r["T"][0][imax] < a["T_max"] * 1.5
    assert a["T_min"] / 1.5 < r["T"][0][imin] < a["T_min"] * 1.5
    assert np.interp(np.log(2e3), np.log(n), r["T"][0]) == pytest.approx(a["T_at_2e3"], rel=0.2)
    # the unstable branch: pressure falls between the two extrema
    assert np.all(np.diff(P[imax:imin + 1]) <= 0)


def test_unshielded_cells_are_in_steady_state():
    # The settled state zeroes the source terms: net heating, H2 and H+ rates vanish
    # against their gross terms (a property of the state, independent of the integrator).
    n, r = _unshielded(n=np.logspace(-1, 3.5, 10))
    p = oracle.default_params(mode=1, flags=oracle.F_CONST_KGR)
    for i in range(n.size):
        cell = dict(n=n[i], chi_pe=1.0, chi_lw=1.0, f_h2=1.0, f_c=1.0, F_lyc=0.0, xi=2e-16, Zg=1.0, Zd=1.0)
        t = oracle.terms(cell, r["T"][0][i], r["xH2"][0][i], r["xHp"][0][i], p)
        gross = n[i] * t["G_total"]
        assert abs(t["H"]) <= 1e-5 * gross, (n[i], t["H"], gross)
        assert r["chg"][0][i] < 1e-4


def test_extrema_scale_with_radiation_and_metallicity():
    a = A["minmax_scaling"]
    assert "linearly" in a["cite"]
    n = np.logspace(-1.5, 4.5, 121)
    _, r = _unshielded(chi0=(1.0, 10.0), Z=(1.0, 1.0), n=n)
    P1, P10 = r["P"][0][r["i_max"][0]], r["P"][1][r["i_max"][1]]
    assert 4.0 < P10 / P1 < 25.0
    Pn1, Pn10 = r["P"][0][r["i_min"][0]], r["P"][1][r["i_min"][1]]
    assert 4.0 < Pn10 / Pn1 < 25.0
    T1, T10 = r["T"][0][r["i_max"][0]], r["T"][1][r["i_max"][1]]
    assert 0.7 < T10 / T1 < 1.4
    _, rz = _unshielded(chi0=(1.0, 1.0), Z=(1.0, 0.1), n=n)
    assert rz["P"][1][rz["i_max"][1]] > rz["P"][0][rz["i_max"][0]]
    assert n[rz["i_max"][1]] >= n[rz["i_max"][0]]


# ------------------------------------------------------------------ shielded curve
@pytest.fixture(scope="module")
def shielded():
    n = np.logspace(-1, 6, 71)
    p = oracle.default_params(mode=1, flags=oracle.F_CONST_KGR, T_cmb=6.0, tau_opt_over_tau_pe=1 / 1.87)
    return n, p, oz.curves(n, [1.0], [2e-16], [1.0], [1.0], p, nchunk=100, shielded=True)


def test_shielded_curve_matches_printed_transitions(shielded):
    a = A["shielded_equilibrium"]
    n, p, r = shielded
    assert np.all(r["status"] == 0)
    x2, xco = r["xH2"][0], r["xCO"][0] / (1.6e-4)
    n_mol = n[np.argmax(x2 > a["xH2_molecular"])]
    n_co = n[np.argmax(xco > a["xCO_over_xC"])]
    assert a["n_molecular"] / 2 < n_mol < a["n_molecular"] * 2
    assert a["n_CO"] / 2 < n_co < a["n_CO"] * 2
    assert r["T"][0][-1] == pytest.approx(a["T_at_1e6"], rel=0.3)
    assert np.all(np.diff(x2) > -1e-6)          # more shielding, more H2


def test_shielded_cr_takes_over_pe_heating(shielded):
    a = A["shielded_equilibrium"]
    n, p, r = shielded
    for i in range(0, n.size, 5):
        chi_pe, chi_lw, f_h2, xi = oz.shielded_fields(n[i], r["xH2"][0][i], 1.0, 2e-16, 1.0)
        cell = dict(n=n[i], chi_pe=chi_pe, chi_lw=chi_lw, f_h2=f_h2, f_c=1.0, F_lyc=0.0, xi=xi, Zg=1.0, Zd=1.0)
        t = oracle.terms(cell, r["T"][0][i], r["xH2"][0][i], r["xHp"][0][i], p)
        ln = np.log10(n[i])
        if ln < a["log10_n_cr_over_pe"] - 0.5:
            assert t["G_pe"] > t["G_cr"], n[i]
        elif ln > a["log10_n_cr_over_pe"] + 0.5:
            assert t["G_cr"] > t["G_pe"], n[i]
        # settled: net heating vanishes against the gross
        assert abs(t["H"]) <= 1e-4 * n[i] * t["G_total"], n[i]
