"""Seeded synthetic inputs for the thermochemistry step (shared by the oracle tests and
the CUDA path; holds none of the step's arithmetic).

Every generator draws from numpy's counter-based Philox stream keyed by the workload
id, so both sides see identical inputs.  The workloads stand in for TIGRESS-like
simulation snapshots, which are not available; the recipes are:

* ``cells_4096``   (id 1): 16^3 independent cells, log n ~ U[-2, 4], log T ~ U[1, 7],
  x_H2 ~ U[0, 0.5], x_H+ ~ U[0, 1 - 2 x_H2], log chi_FUV ~ U[-1, 3] with chi_PE = chi_LW
  = chi_FUV, f_shld,H2 ~ U[1e-6, 1], f_shld,C = 1, no ionising flux, xi = 2e-16 s^-1,
  Z' = 1.
* ``slab``         (id 2): lognormal n (median 1 cm^-3, sigma_ln = 1.5); T from a
  two-phase P/k = 3000 K cm^-3 relation with 20% lognormal scatter; x_H2 rising to 0.5
  above n ~ 100; six ray columns per cell log-uniform in [1e18, 1e23] cm^-2 mapped to
  chi_PE, chi_LW, the H2 self-shielding factor and the attenuated CR rate.
* ``stiff``        (id 3): the slab plus 32 spheres (radius 4..16 cells): 16 H II
  regions with ionising flux 1e7..1e11 cm^-2 s^-1 falling as r^-2, 16 SN-remnant
  interiors at 1e6..1e8 K and 1% of the ambient density.
* ``boxes``        (id 5): 48 boxes of 32^3..128^3 cells with per-box Z', chi and xi
  scales and the ``cells_4096`` distributions inside.
* ``training_samples`` (id 4): slab-distributed states with Z' in [0.1, 3] and
  step lengths log-uniform in [1e-3, 1] x 1e4 yr.

The upstream radiation quantities of the slab (dust attenuation, Draine & Bertoldi
H2 self-shielding, Eq. e:fshld_H2_DB, effective-column CR attenuation, Eqs.
e:tau_eff and e:cratt) are the paper's Sec. 5 relations, which sit before the step
and are inputs to it.
"""
from __future__ import annotations

import numpy as np

YEAR_S = 3.15576e7
DT_1E4YR = 1e4 * YEAR_S

SIGMA_D_PE = 1.0e-21   # cm^2 per H (Sec. 5.3, used for N_eff and PE attenuation)
SIGMA_D_LW = 1.5e-21   # cm^2 per H (Sec. 2.4, LW absorption)
N0_CR = 9.35e20        # Eq. e:cratt
XI0 = 2.0e-16

KEYS = ("n", "chi_pe", "chi_lw", "f_h2", "f_c", "F_lyc", "xi", "Zg", "Zd", "T", "xH2", "xHp")


def _rng(key: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(key), int(sub)]))


def f_shld_h2_db(N_h2, b5=3.0):
    """Draine & Bertoldi (1996) H2 self-shielding, Eq. e:fshld_H2_DB (b5 = 3)."""
    x = np.asarray(N_h2, dtype=np.float64) / 5e14
    s = np.sqrt(1.0 + x)
    return 0.965 / (1.0 + x / b5) ** 2 + 0.035 / s * np.exp(-8.5e-4 * s)


def xi_attenuated(chi_pe, chi0=1.0, xi0=XI0, Zd=1.0):
    """CR attenuation from the effective column, Eqs. e:tau_eff and e:cratt."""
    tau = -np.log(np.clip(np.asarray(chi_pe) / chi0, 1e-300, 1.0))
    Neff = tau / (SIGMA_D_PE * Zd)
    return np.where(Neff <= N0_CR, xi0, xi0 * N0_CR / np.maximum(Neff, N0_CR))


def cells_4096(n: int = 4096, key: int = 1, chi_scale: float = 1.0, xi: float = 2e-16, Z: float = 1.0) -> dict:
    g = _rng(key)
    lg_n = g.uniform(-2.0, 4.0, n)
    lg_T = g.uniform(1.0, 7.0, n)
    xH2 = g.uniform(0.0, 0.5, n)
    xHp = g.uniform(0.0, 1.0, n) * (1.0 - 2.0 * xH2)
    lg_chi = g.uniform(-1.0, 3.0, n)
    fsh = g.uniform(1e-6, 1.0, n)
    chi = chi_scale * 10.0 ** lg_chi
    return dict(n=10.0 ** lg_n, T=10.0 ** lg_T, xH2=xH2, xHp=xHp, chi_pe=chi, chi_lw=chi.copy(), f_h2=fsh,
                f_c=np.ones(n), F_lyc=np.zeros(n), xi=np.full(n, xi), Zg=np.full(n, Z), Zd=np.full(n, Z))


def slab(side: int = 128, key: int = 2, chi0: float = 1.0, Z: float = 1.0, ncell: int | None = None) -> dict:
    n_cells = side ** 3 if ncell is None else int(ncell)
    g = _rng(key)
    n = np.exp(g.normal(0.0, 1.5, n_cells))
    xH2 = 0.5 / (1.0 + (30.0 / n) ** 2)
    T = 3000.0 / ((1.1 - xH2) * n) * np.exp(0.2 * g.normal(0.0, 1.0, n_cells))
    T = np.clip(T, 10.0, 1e7)
    xHp = np.minimum(0.026 / np.sqrt(n), 1.0 - 2.0 * xH2)
    N = 10.0 ** g.uniform(18.0, 23.0, (6, n_cells))
    att_pe = np.exp(-SIGMA_D_PE * Z * N)
    att_lw = np.exp(-SIGMA_D_LW * Z * N)
    chi_pe = chi0 * att_pe.mean(axis=0)
    chi_lw = chi0 * att_lw.mean(axis=0)
    wsum = att_lw.sum(axis=0)
    fsh = (att_lw * f_shld_h2_db(xH2[None, :] * N)).sum(axis=0) / np.maximum(wsum, 1e-300)
    fsh = np.where(wsum > 0, fsh, f_shld_h2_db(xH2 * N.max(axis=0)))
    xi = xi_attenuated(chi_pe, chi0, XI0, Z)
    del N, att_pe, att_lw
    return dict(n=n, T=T, xH2=xH2, xHp=xHp, chi_pe=chi_pe, chi_lw=chi_lw, f_h2=fsh, f_c=np.ones(n_cells),
                F_lyc=np.zeros(n_cells), xi=xi, Zg=np.full(n_cells, Z), Zd=np.full(n_cells, Z))


def stiff(side: int = 256, key: int = 3, nsph: int = 32) -> dict:
    c = slab(side=side, key=key)
    g = _rng(key, 1)
    idx = np.arange(side)
    for s in range(nsph):
        r = int(g.integers(4, 17))
        cen = g.integers(0, side, 3)
        lo = np.maximum(cen - r, 0)
        hi = np.minimum(cen + r + 1, side)
        zz, yy, xx = np.meshgrid(idx[lo[0]:hi[0]], idx[lo[1]:hi[1]], idx[lo[2]:hi[2]], indexing="ij")
        d = np.sqrt((zz - cen[0]) ** 2 + (yy - cen[1]) ** 2 + (xx - cen[2]) ** 2)
        m = d <= r
        flat = (zz[m] * side + yy[m]) * side + xx[m]
        if s < nsph // 2:   # H II region
            F0 = 10.0 ** g.uniform(7.0, 11.0)
            c["F_lyc"][flat] = F0 / np.maximum(d[m], 1.0) ** 2
            c["T"][flat] = 1e4
            c["xH2"][flat] = 0.0
            c["xHp"][flat] = 0.5
        else:               # SN remnant interior
            T0 = 10.0 ** g.uniform(6.0, 8.0)
            c["T"][flat] = T0
            c["n"][flat] *= 0.01
            c["xH2"][flat] = 0.0
            c["xHp"][flat] = 1.0
    return c


BOX_SIDES = (32, 48, 64, 96, 128)


def boxes(nbox: int = 48, key: int = 5):
    """List of (cells, scalars) for the batched sweep; scalars holds Z', chi scale, xi."""
    g = _rng(key)
    out = []
    for b in range(nbox):
        side = int(g.choice(BOX_SIDES))
        Z = float(10.0 ** g.uniform(-1.0, np.log10(3.0)))
        chis = float(10.0 ** g.uniform(-1.0, 2.0))
        xi = float(10.0 ** g.uniform(-17.0, -15.0))
        cells = cells_4096(n=side ** 3, key=1000 + b, chi_scale=chis, xi=xi, Z=Z)
        out.append((cells, dict(side=side, Z=Z, chi_scale=chis, xi=xi)))
    return out


def training_samples(n: int, key: int = 4) -> dict:
    """Slab-distributed states with Z' log-uniform in [0.1, 3] and dt log-uniform in
    [1e-3, 1] x 1e4 yr; dt is returned under key 'dt'."""
    c = slab(key=key, ncell=n)
    g = _rng(key, 7)
    Z = 10.0 ** g.uniform(-1.0, np.log10(3.0), n)
    c["Zg"] = Z
    c["Zd"] = Z.copy()
    c["dt"] = DT_1E4YR * 10.0 ** g.uniform(-3.0, 0.0, n)
    return c


def subset(cells: dict, idx) -> dict:
    return {k: (np.asarray(v)[idx] if np.ndim(v) else v) for k, v in cells.items()}
