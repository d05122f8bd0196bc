"""Pins of the oracle's time integration: invariants that hold by construction,
closed-form steady states, convergence to a tight-tolerance RK45 reference, and the
shape of the paper's unshielded equilibrium curve (Sec. 7.1.1)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthgen

HERE = os.path.dirname(os.path.abspath(__file__))
A = json.load(open(os.path.join(HERE, "golden", "paper_anchors.json")))
YR = 3.15576e7
DT = synthgen.DT_1E4YR


@pytest.fixture(scope="module")
def config1_both_modes():
    c = synthgen.cells_4096()
    return c, {m: oracle.step(c, DT, oracle.default_params(mode=m)) for m in (0, 1)}


@pytest.mark.parametrize("mode", [0, 1])
def test_hydrogen_bounds_and_status(config1_both_modes, mode):
    c, R = config1_both_modes
    r = R[mode]
    assert np.all(r["status"] == 0)
    assert np.all(np.isfinite(r["T"])) and np.all(r["T"] > 0)
    xH = 1.0 - 2.0 * r["xH2"] - r["xHp"]
    assert r["xH2"].min() >= 0.0 and r["xHp"].min() >= 0.0
    assert xH.min() >= -1e-14          # H nuclei conserved, x_H >= 0 up to rounding
    assert r["xH2"].max() <= 0.5 and r["xHp"].max() <= 1.0 + 1e-14


@pytest.mark.parametrize("mode", [0, 1])
def test_carbon_oxygen_conservation_and_neutrality(config1_both_modes, mode):
    c, R = config1_both_modes
    r = R[mode]
    idx = np.arange(0, 4096, 37)
    for i in idx:
        cell = {k: float(c[k][i]) for k in oracle.CELL_KEYS}
        t = oracle.terms(cell, r["T"][i], r["xH2"][i], r["xHp"][i])
        xCtot, xOtot = 1.6e-4 * cell["Zg"], 3.2e-4 * cell["Zg"]
        assert t["xC"] + t["xCp"] + t["xCO"] == pytest.approx(xCtot, rel=1e-13)
        assert t["xO"] + t["xOp"] + t["xCO"] == pytest.approx(xOtot, rel=1e-13)
        for k in ("xC", "xCp", "xCO", "xO", "xOp"):
            assert t[k] >= -1e-20
        assert t["xOp"] == pytest.approx(xOtot * r["xHp"][i], rel=1e-14)
        if r["T"][i] < 1e4:   # S(T) < 1e-5: Eq. e:xEL holds on its own
            lhs = r["xHp"][i] + t["xCp"] + t["xOp"] + t["xMHp"]
            assert t["xe"] == pytest.approx(lhs, rel=1e-5)


def _steady(cells, params, repeats, dt=1e13 * YR):
    """Integrates to steady state.  Mode 0 lags x_e by one substep, so its final long
    substep leaves one fixed-point iteration undone; repeating the step converges it."""
    c = dict(cells)
    for _ in range(repeats):
        r = oracle.step(c, dt, params)
        c.update(T=r["T"], xH2=r["xH2"], xHp=r["xHp"])
    return r


@pytest.mark.parametrize("mode,repeats", [(0, 40), (1, 8)])
def test_photoionisation_recombination_balance(mode, repeats):
    # x_H2 = 0, Z' = 0 (no C, O, grains), xi = 0: zeta (1-x) + k_ci n x (1-x) = alpha n x^2
    # (Eq. e:HII with x_e = x_H+), a quadratic with one positive root.
    F = np.array([1e5, 1e7, 1e9, 1e11])
    cells = dict(n=np.array([0.1, 1.0, 10.0, 100.0]), T=8000.0, xH2=0.0, xHp=np.full(4, 0.3), chi_pe=0.0,
                 chi_lw=0.0, f_h2=1.0, f_c=1.0, F_lyc=F, xi=0.0, Zg=0.0, Zd=0.0)
    r = _steady(cells, oracle.default_params(mode=mode, flags=oracle.F_FREEZE_T), repeats)
    for i in range(4):
        n = cells["n"][i]
        t = oracle.terms({k: (cells[k][i] if np.ndim(cells[k]) else cells[k]) for k in oracle.CELL_KEYS},
                         r["T"][i], 0.0, r["xHp"][i])
        z, a, k = 3.1e-18 * F[i], t["arr"], t["kci"]
        qa, qb, qc = (a + k) * n, z - k * n, -z
        x = (-qb + math.sqrt(qb * qb - 4 * qa * qc)) / (2 * qa)
        assert r["xHp"][i] == pytest.approx(x, rel=1e-9)
        assert r["xe"][i] == pytest.approx(r["xHp"][i], rel=1e-9)


@pytest.mark.parametrize("mode", [0, 1])
def test_h2_formation_photodissociation_balance_no_cr(mode):
    # xi = 0, no LyC, T = 100 K: x_H+ stays 0 and Eq. e:HH gives k n (1 - 2x) = zeta_pd x.
    chi = np.array([0.01, 0.1, 1.0, 10.0])
    fsh = np.array([1e-4, 1e-3, 1e-2, 0.5])
    cells = dict(n=100.0, T=100.0, xH2=np.full(4, 0.1), xHp=0.0, chi_pe=chi, chi_lw=chi, f_h2=fsh, f_c=1.0,
                 F_lyc=0.0, xi=0.0, Zg=1.0, Zd=1.0)
    p = oracle.default_params(mode=mode, flags=oracle.F_FREEZE_T | oracle.F_CONST_KGR)
    r = _steady(cells, p, 3)
    kn = 3e-17 * 100.0
    zpd = 5.7e-11 * chi * fsh
    x = kn / (2 * kn + zpd)
    np.testing.assert_allclose(r["xH2"], x, rtol=1e-9)
    assert np.all(r["xHp"] == 0.0)


@pytest.mark.parametrize("mode,repeats", [(0, 40), (1, 8)])
def test_h2_balance_with_cosmic_rays(mode, repeats):
    # Eq. e:HH with Eq. eq:H2_cr and no photo-/collisional terms: a quadratic in x = x_H2
    # given the steady x_+ = x_H+:
    # k n (1 - 2x - x_+) = (1.65 * 2 xi (2.3 x + 1.5 (1 - 2x - x_+)) + zeta_pd) x.
    chi = np.array([1e-4, 1e-3, 1e-2])
    cells = dict(n=300.0, T=50.0, xH2=np.full(3, 0.2), xHp=np.full(3, 1e-4), chi_pe=chi, chi_lw=chi, f_h2=1e-3,
                 f_c=1.0, F_lyc=0.0, xi=2e-16, Zg=1.0, Zd=1.0)
    p = oracle.default_params(mode=mode, flags=oracle.F_FREEZE_T | oracle.F_CONST_KGR)
    r = _steady(cells, p, repeats)
    kn = 3e-17 * 300.0
    a1 = 1.65 * 2.0 * 2e-16
    for i in range(3):
        xp = r["xHp"][i]
        z = 5.7e-11 * chi[i] * 1e-3
        B = 1.5 * a1 * (1 - xp) + z + 2 * kn
        C = kn * (1 - xp)
        x = (B - math.sqrt(B * B - 4 * 0.7 * a1 * C)) / (2 * 0.7 * a1)
        assert r["xH2"][i] == pytest.approx(x, rel=1e-9)


def test_dust_temperature_closed_form():
    # With negligible gas-dust coupling (n -> 0), Eq. eq:dust_en reduces to
    # B z (z^2 - T_cmb^4) = Gamma_d with z = T_d^2 and B = 2e-27 Z'_d c a: a cubic.
    for chi in (0.1, 1.0, 30.0, 1e3):
        cell = dict(n=1e-12, chi_pe=chi, chi_lw=chi)
        t = oracle.terms(cell, 100.0, 0.0, 0.0)
        P = oracle.prepared(cell)
        B = 2e-27 * 1.0 * 2.99792458e10 * 7.57e-15
        roots = np.roots([B, 0.0, -B * 2.73 ** 4, -P["Gd"]])
        z = max(r.real for r in roots if abs(r.imag) < 1e-12 and r.real > 0)
        assert t["Td"] == pytest.approx(math.sqrt(z), rel=1e-10)


def test_rk45_convergence_order():
    # The scheme of Sec. 6.1 is first order in the substep length: shrinking the limiter
    # 0.1 -> 0.01 -> 0.001 must approach a tight RK45 solution of the same ODE/algebraic
    # system with observed order ~1 (non-stiff cells, dt = 1e3 yr).
    g = np.random.default_rng(11)
    m = 40
    cells = dict(n=10 ** g.uniform(-1, 1, m), T=10 ** g.uniform(1.7, 3.9, m), xH2=g.uniform(0, 0.3, m),
                 xHp=g.uniform(1e-3, 0.2, m), chi_pe=10 ** g.uniform(-1, 0.5, m), f_h2=g.uniform(0.05, 1, m),
                 f_c=1.0, F_lyc=0.0, xi=2e-16, Zg=1.0, Zd=1.0)
    cells["chi_lw"] = cells["chi_pe"]
    dt = 1e3 * YR
    ref = np.array([oracle.rk45({k: (cells[k][i] if np.ndim(cells[k]) else cells[k]) for k in oracle.CELL_KEYS},
                                cells["T"][i], cells["xH2"][i], cells["xHp"][i], dt)[0] for i in range(m)])
    for mode in (0, 1):
        errs = []
        for lim in (0.1, 0.01, 0.001):
            r = oracle.step(cells, dt, oracle.default_params(mode=mode, limiter=lim))
            e = np.max(np.abs(r["T"] - ref[:, 0]) / ref[:, 0]) + np.max(np.abs(r["xHp"] - ref[:, 2]))
            errs.append(e)
        order = [math.log10(errs[i] / errs[i + 1]) for i in range(2)]
        assert errs[2] < 2e-3
        assert 0.6 < order[1] < 1.5, (mode, errs)


def test_mode_a_and_b_agree_as_substeps_shrink():
    c = synthgen.subset(synthgen.cells_4096(), slice(0, 256))
    ra = oracle.step(c, DT, oracle.default_params(mode=0, limiter=0.002))
    rb = oracle.step(c, DT, oracle.default_params(mode=1, limiter=0.002))
    assert np.median(np.abs(ra["T"] - rb["T"]) / rb["T"]) < 3e-3


def test_unshielded_equilibrium_curve_shape():
    # Sec. 7.1.1 (chi0 = 1, xi = 2e-16, Z' = 1, unshielded, constant k_gr as in Sec. 7):
    # a warm branch up to P_max near n ~ 1, an unstable branch with dlogP/dlogn < 0, a
    # cold branch from P_min near n ~ 10, and T = 32 K at n = 2e3.  Closures are not
    # the paper's exact fits, so the tolerances are loose (factor ~2).
    a = A["unshielded_equilibrium"]
    n = np.logspace(-1, 3.5, 91)
    N = n.size
    cells = dict(n=n, T=np.full(N, 3000.0), xH2=np.zeros(N), xHp=np.full(N, 1e-2), chi_pe=1.0, chi_lw=1.0,
                 f_h2=1.0, f_c=1.0, F_lyc=0.0, xi=2e-16, Zg=1.0, Zd=1.0)
    p = oracle.default_params(flags=oracle.F_CONST_KGR)
    r = oracle.step(cells, 2e8 * YR, p)
    P = (1.1 + r["xe"] - r["xH2"]) * n * r["T"]
    lp = np.log(P)
    d = np.diff(lp) / np.diff(np.log(n))
    imax = int(np.argmax(d < 0))                      # first point where P decreases
    imin = imax + int(np.argmax(d[imax:] > 0))        # then where it rises again
    assert imin > imax
    Pmax, Pmin = P[imax], P[imin]
    assert a["Pmax_k"] / 2 < Pmax < a["Pmax_k"] * 2
    assert a["Pmin_k"] / 2 < Pmin < a["Pmin_k"] * 2
    assert a["n_max"] / 2 < n[imax] < a["n_max"] * 2
    assert a["n_min"] / 2.5 < n[imin] < a["n_min"] * 2
    assert a["T_max"] / 1.5 < r["T"][imax] < a["T_max"] * 1.5
    assert a["T_min"] / 1.5 < r["T"][imin] < a["T_min"] * 1.5
    T2e3 = np.interp(np.log(2e3), np.log(n), r["T"])
    assert T2e3 == pytest.approx(a["T_at_2e3"], rel=0.2)


def _stiff_class(kind, m, seed):
    g = np.random.default_rng(seed)
    if kind == "hot":          # collisionally ionised gas cooling from 1e5-1e7 K
        c = dict(n=10 ** g.uniform(-2, 1, m), T=10 ** g.uniform(5, 7, m), xH2=np.zeros(m),
                 xHp=g.uniform(0.5, 1.0, m), chi_pe=10 ** g.uniform(-1, 1, m), f_h2=np.ones(m), F_lyc=np.zeros(m))
    elif kind == "ionised":    # photoionised gas, F_LyC = 1e7-1e10 cm^-2 s^-1
        c = dict(n=10 ** g.uniform(0, 2, m), T=10 ** g.uniform(3.7, 4.2, m), xH2=np.zeros(m),
                 xHp=g.uniform(0.01, 0.99, m), chi_pe=10 ** g.uniform(0, 2, m), f_h2=np.ones(m),
                 F_lyc=10 ** g.uniform(7, 10, m))
    else:                      # dense shielded molecular gas
        c = dict(n=10 ** g.uniform(2, 4, m), T=10 ** g.uniform(1, 2.3, m), xH2=g.uniform(0.3, 0.5, m),
                 xHp=10 ** g.uniform(-7, -4, m), chi_pe=10 ** g.uniform(-3, -1, m), f_h2=10 ** g.uniform(-6, -2, m),
                 F_lyc=np.zeros(m))
    c.update(f_c=1.0, xi=2e-16, Zg=1.0, Zd=1.0)
    c["chi_lw"] = c["chi_pe"]
    return c


@pytest.mark.parametrize("kind", ["hot", "ionised", "molecular"])
def test_rk45_convergence_stiff_classes(kind):
    # 100 cells per class (hot 1e5-1e7 K, photoionised, dense molecular), one step of
    # dt = 1e4 yr: both schemes approach the tight RK45 solution of the same
    # differential-algebraic system at first order as the limiter shrinks
    # 0.01 -> 0.001 -> 0.0001.  The order is taken on the summed error over the cells
    # (and on the median cell): a few cold cells are still pre-asymptotic at 1e-3.
    from concurrent.futures import ThreadPoolExecutor
    m = 100
    c = _stiff_class(kind, m, 5)
    dt = 1e4 * YR

    def one(i):
        cell = {k: (c[k][i] if np.ndim(c[k]) else c[k]) for k in oracle.CELL_KEYS}
        return oracle.rk45(cell, c["T"][i], c["xH2"][i], c["xHp"][i], dt)[0]

    with ThreadPoolExecutor(8) as ex:
        ref = np.array(list(ex.map(one, range(m))))
    for mode in (0, 1):
        errs = []
        for lim in (0.01, 0.001, 0.0001):
            r = oracle.step(c, dt, oracle.default_params(mode=mode, limiter=lim))
            assert np.all((r["status"] & (oracle.ST_NEWTON | oracle.ST_NONFINITE)) == 0)
            errs.append(np.abs(r["T"] - ref[:, 0]) / ref[:, 0] + np.abs(r["xH2"] - ref[:, 1]) +
                        np.abs(r["xHp"] - ref[:, 2]))
        errs = np.array(errs)
        l1 = errs.sum(axis=1)
        assert errs[2].max() < 2e-3, (kind, mode, errs.max(axis=1))
        for a, b in ((0, 1), (1, 2)):
            assert 0.85 < math.log10(l1[a] / l1[b]) < 1.15, (kind, mode, l1)
        assert 0.85 < np.median(np.log10(errs[1] / errs[2])) < 1.15, (kind, mode)
