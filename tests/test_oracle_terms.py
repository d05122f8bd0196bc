"""Pins of the oracle's individual printed terms of Secs. 3-4 against hand evaluations of
the paper's formulas (tests/golden/paper_anchors.json, entries "hand_*", each with its
citation and the arithmetic written out).

Each test isolates one term through the oracle's term dump (oracle.terms) at a state
chosen so that a wrong constant, exponent or energy in that term changes the result by
far more than the tolerance: Lyman-alpha cooling (Eq. e:k_lya), the H2 formation,
pumping and dissociation heating with their n_crit (Eqs. e:Gamma_H2form/pump/diss),
the cooling sigmoid S(T), gas-dust cooling (Eq. eq:gas-dust), photoionization heating
(Eqs. eq:photoion_heat, eq:photoion_heat_H2), the energies of collisional ionisation
and dissociation cooling (Eqs. e:Lambda_ci_H, e:Lambda_cd_H2), nebular cooling (Eq.
e:Lambda_neb), the CO critical density (Eq. e:CO_fit) and the H2 photodissociation rate
(Eq. eq:H2_pd).
"""
import json
import math
import os

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
A = json.load(open(os.path.join(HERE, "golden", "paper_anchors.json")))
EV = 1.602176634e-12


def _terms(T, xH2=0.0, xHp=0.0, params=None, Td=-1.0, **cell):
    return oracle.terms(cell, T, xH2, xHp, params, Td=Td)


@pytest.mark.parametrize("key", ["hand_lya_T1e4", "hand_lya_T2e4"])
def test_lyman_alpha_cooling(key):
    a = A[key]
    for xH2, xHp in ((0.0, 0.3), (0.1, 0.05)):
        t = _terms(a["T"], xH2=xH2, xHp=xHp, n=10.0)
        xH = 1.0 - 2.0 * xH2 - xHp
        assert t["L_lya"] / (xH * t["xe"]) == pytest.approx(a["value"], rel=1e-9)


def test_cooling_sigmoid():
    a = A["hand_sigmoid_S"]
    for T, v in zip(a["T"], a["value"]):
        assert _terms(T, xHp=0.5)["S"] == pytest.approx(v, rel=1e-9)


@pytest.mark.parametrize("i", [0, 1])
def test_gas_dust_cooling(i):
    c = A["hand_gas_dust"]["cases"][i]
    t = _terms(c["T"], n=1e3, Zd=c["Zd"], Td=c["Td"])
    assert t["Td"] == c["Td"]
    assert t["L_gd"] == pytest.approx(c["value"], rel=1e-12)


def test_h2_heating_terms_and_critical_density():
    a = A["hand_h2_heating"]
    s = a["state"]
    cell = dict(chi_lw=s["chi_lw"], chi_pe=s["chi_lw"], f_h2=s["f_h2"])
    # photodissociation heating: 0.4 eV per dissociation at any density
    for n in (1e-3, 1.0, 1e9):
        t = _terms(s["T"], s["xH2"], s["xHp"], n=n, **cell)
        assert t["zpd"] == pytest.approx(s["zeta_pd"], rel=1e-12)
        assert t["G_h2pd"] / (t["zpd"] * s["xH2"]) == pytest.approx(a["pd_per_zpd_xH2_eV"] * EV, rel=1e-12)
    # low- and high-density limits of the de-excitation factor 1/(1 + n_crit/n)
    lo = _terms(s["T"], s["xH2"], s["xHp"], n=1e-4, **cell)
    hi = _terms(s["T"], s["xH2"], s["xHp"], n=1e16, **cell)
    assert lo["G_h2form"] / (lo["kgr"] * 1e-4 * s["xH"]) == pytest.approx(a["form_per_kgr_n_xH_eV"]["n_to_0"] * EV, rel=1e-9)
    assert lo["G_h2pump"] / (lo["zpd"] * s["xH2"]) == pytest.approx(0.0, abs=1e-9 * EV)
    assert hi["G_h2form"] / (hi["kgr"] * 1e16 * s["xH"]) == pytest.approx(a["form_per_kgr_n_xH_eV"]["n_to_inf"] * EV, rel=1e-6)
    assert hi["G_h2pump"] / (hi["zpd"] * s["xH2"]) == pytest.approx(a["pump_per_zpd_xH2_eV"]["n_to_inf"] * EV, rel=1e-6)
    # at n = n_crit (A_eff = 2e-7 s^-1 plus zeta_pd over the collisional de-excitation
    # rate per density) the factor is exactly 1/2; and one density above it
    for c in a["at_n"]:
        t = _terms(s["T"], s["xH2"], s["xHp"], n=c["n"], **cell)
        assert t["G_h2form"] / (t["kgr"] * c["n"] * s["xH"]) == pytest.approx(c["form_eV"] * EV, rel=1e-9)
        assert t["G_h2pump"] / (t["zpd"] * s["xH2"]) == pytest.approx(c["pump_eV"] * EV, rel=1e-9)


def test_photoionization_heating():
    a = A["hand_photoion_heating"]
    F = 1e9
    P = oracle.prepared(dict(F_lyc=F))
    assert P["zpiH"] == pytest.approx(a["sigma_pi_H"] * F, rel=1e-15)
    assert P["zpiH2"] == pytest.approx(a["sigma_pi_H2"] * F, rel=1e-15)
    # atomic gas: only the H term; molecular gas: only the H2 term
    t = _terms(8000.0, xH2=0.0, xHp=0.4, n=1.0, F_lyc=F)
    assert t["G_pi"] / (0.6 * P["zpiH"]) == pytest.approx(a["q_pi_H_eV"] * EV, rel=1e-12)
    t = _terms(100.0, xH2=0.5, xHp=0.0, n=1.0, F_lyc=F)
    assert t["G_pi"] / (0.5 * P["zpiH2"]) == pytest.approx(a["q_pi_H2_eV"] * EV, rel=1e-12)


def test_collisional_ionisation_and_dissociation_energies():
    a = A["hand_ci_cd_energies"]
    for T, xH2, xHp in ((2e4, 0.0, 0.3), (5e4, 0.2, 0.1), (3e3, 0.3, 0.01)):
        t = _terms(T, xH2=xH2, xHp=xHp, n=10.0)
        xH = 1.0 - 2.0 * xH2 - xHp
        assert t["L_ci"] / (xH * t["xe"] * t["kci"]) == pytest.approx(a["ci_eV"] * EV, rel=1e-12)
        if xH2 > 0:
            assert t["L_cd"] / (xH2 * (xH * t["kcdH"] + xH2 * t["kcdH2"])) == pytest.approx(a["cd_eV"] * EV, rel=1e-12)


@pytest.mark.parametrize("i", [0, 1, 2])
def test_nebular_cooling(i):
    c = A["hand_neb"]["cases"][i]
    T = c["T4"] * 1e4
    for n, Zg in ((1e-3, 1.0), (300.0, 0.5)):
        t = _terms(T, xHp=0.9, n=n, Zg=Zg)
        ne2 = t["xe"] * n / 100.0
        expect = Zg * t["xe"] * 0.9 * c["A"] / (1.0 + 0.12 * ne2 ** c["exponent"])
        assert t["L_neb"] == pytest.approx(expect, rel=1e-9)


@pytest.mark.parametrize("i", [0, 1, 2])
def test_co_critical_density(i):
    c = A["hand_nco_crit"]["cases"][i]
    P = oracle.prepared(dict(chi_lw=c["chi_lw"], chi_pe=c["chi_lw"], xi=c["xi"], Zd=c["Zd"]))
    assert math.exp(P["lnCO"]) == pytest.approx(c["value"], rel=1e-9)


def test_h2_photodissociation_rate():
    c = A["hand_zeta_pd"]["cases"][0]
    P = oracle.prepared(dict(chi_lw=c["chi_lw"], f_h2=c["f_h2"]))
    assert P["zpd"] == pytest.approx(c["value"], rel=1e-15)
