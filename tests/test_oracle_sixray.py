"""Pins of the oracle's six-ray fields (Secs. 5.2, 5.3): brute-force columns, photon
conservation along a ray, the transparent limit, symmetry, and the centre of a uniform
cube, where the six columns are equal and the effective column and the H2 shielding
reduce to closed forms."""
import numpy as np
import pytest

from oracle import sixray as sr

PC = 3.0856775814913673e18


def _brute_columns(q, dx):
    nz, ny, nx = q.shape
    out = [np.zeros_like(q) for _ in range(6)]
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                out[0][k, j, i] = sum(q[k, j, a] for a in range(0, i)) * dx
                out[1][k, j, i] = sum(q[k, j, a] for a in range(i + 1, nx)) * dx
                out[2][k, j, i] = sum(q[k, a, i] for a in range(0, j)) * dx
                out[3][k, j, i] = sum(q[k, a, i] for a in range(j + 1, ny)) * dx
                out[4][k, j, i] = sum(q[a, j, i] for a in range(0, k)) * dx
                out[5][k, j, i] = sum(q[a, j, i] for a in range(k + 1, nz)) * dx
    return out


def test_columns_match_brute_force():
    rng = np.random.default_rng(0)
    q = rng.lognormal(0.0, 1.5, (3, 4, 5))
    for a, b in zip(sr.ray_columns(q, 2.0), _brute_columns(q, 2.0)):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-12 * b.max())


def test_photon_conservation_along_a_line():
    # 1 x 1 x nx grid: the y and z rays only cross the cell itself.  Photons deposited
    # by the two x rays over the line equal those entering minus those leaving:
    # sum_k dtau_k g_k (e^-tau_in+ + e^-tau_in-) = 2 (1 - e^-tau_tot).
    rng = np.random.default_rng(1)
    n = rng.lognormal(2.0, 1.0, (1, 1, 200))
    dx = 0.3 * PC
    r = sr.sixray(n, np.zeros_like(n), dx, chi0=1.0, Zd=1.0)
    dtau = sr.SIGMA_PE * n * dx
    g = sr.cell_average(dtau)
    x_rays = 6.0 * r["chi_pe"] - 4.0 * g
    lhs = np.sum(dtau * x_rays)
    rhs = 2.0 * (1.0 - np.exp(-dtau.sum()))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_transparent_limit():
    n = np.full((4, 5, 6), 1e-12)
    r = sr.sixray(n, np.full_like(n, 0.3), 1.0 * PC, chi0=3.0, xi0=2e-16, Zd=1.0)
    np.testing.assert_allclose(r["chi_pe"], 3.0, rtol=1e-12)
    np.testing.assert_allclose(r["chi_lw"], 3.0, rtol=1e-12)
    np.testing.assert_allclose(r["f_h2"], 0.965 + 0.035 * np.exp(-8.5e-4), rtol=1e-6)
    assert np.all(r["xi"] == 2e-16)


def test_axis_symmetry():
    rng = np.random.default_rng(2)
    n = rng.lognormal(1.0, 1.0, (6, 7, 8))
    x = rng.uniform(0.0, 0.5, n.shape)
    dx = 2.0 * PC
    r = sr.sixray(n, x, dx)
    rt = sr.sixray(np.transpose(n, (0, 2, 1)).copy(), np.transpose(x, (0, 2, 1)).copy(), dx)   # swap x and y
    rm = sr.sixray(n[:, :, ::-1].copy(), x[:, :, ::-1].copy(), dx)                               # mirror x
    for k in ("chi_pe", "chi_lw", "f_h2", "N_eff"):
        np.testing.assert_allclose(np.transpose(rt[k], (0, 2, 1)), r[k], rtol=1e-12)
        np.testing.assert_allclose(rm[k][:, :, ::-1], r[k], rtol=1e-12)


def test_uniform_cube_centre_closed_forms():
    # Centre of a uniform cube of side L (odd cell count): all six columns are
    # n (L - dx)/2, so the effective column tends to n L / 2 as the cells thin (the
    # in-cell average contributes dtau/2 to second order) and, with no dust, the H2
    # shielding factor is the printed function at the column to the centre, x n L / 2.
    L, n0, xh2 = 20.0 * PC, 30.0, 0.2
    err = {}
    for m in (25, 51, 101):
        n = np.full((m, m, m), n0)
        dx = L / m
        r = sr.sixray(n, np.full_like(n, xh2), dx, chi0=1.0, xi0=2e-16, Zd=1.0)
        c = m // 2
        err[m] = r["N_eff"][c, c, c] / (n0 * L / 2) - 1.0
        assert abs(err[m]) < 3e-5 * (101 / m) ** 2
        assert r["xi"][c, c, c] == pytest.approx(2e-16 * min(1.0, sr.N0_CR / r["N_eff"][c, c, c]), rel=1e-12)
    # second-order convergence in the cell size
    assert err[25] / err[51] == pytest.approx((51 / 25) ** 2, rel=0.05)
    assert err[51] / err[101] == pytest.approx((101 / 51) ** 2, rel=0.05)
    r0 = sr.sixray(n, np.full_like(n, xh2), dx, Zd=0.0)
    assert r0["f_h2"][c, c, c] == pytest.approx(float(sr.f_shld_h2(xh2 * n0 * L / 2)), rel=1e-12)
    assert np.all(r0["xi"] == 2e-16)


def test_deep_cells_stay_finite():
    n = np.full((3, 3, 400), 1e4)
    r = sr.sixray(n, np.full_like(n, 0.5), 10.0 * PC)
    assert np.all(np.isfinite(r["f_h2"])) and np.all(np.isfinite(r["N_eff"]))
    assert np.all(r["chi_pe"] >= 0.0) and np.all(r["f_h2"] > 0.0)
