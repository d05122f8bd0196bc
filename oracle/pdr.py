"""Plane-parallel PDR slabs and the HI-to-H2 transition column (Secs. 7.2, 7.3), oracle
side.

TEST INFRASTRUCTURE ONLY: the plain statement of the slab driver the library runs on the
GPU (tc_pdr).  Only tests/ and bench.py's CPU legs may call it; it shares no code with
the library.

A uniform-density slab of `ncell` cells of size dx is lit from its surface (cell 0) by
a beamed FUV field of normalised intensity chi0 at normal incidence.  A cell whose near
face lies behind a column N = sum of n_H dx over the cells in front of it sees, averaged
over the cell (Eq. e:Erad with a single ray),

    chi_j = chi0 exp(-sigma_j N) g(sigma_j n_H dx),   g(t) = (1 - e^-t)/t,   j = PE, LW,

the H2 self-shielding factor of Eq. e:fshld_H2_DB at the H2 column to its centre, and
the CR rate of Eq. e:cratt with N_eff the perpendicular column to its centre, N + 0.5
n_H dx.  The slab is evolved in `nchunk` chunks of t_end/nchunk: the fields are computed
from the current x_H2 at the start of each chunk and held over it (the radiation is held
over a hydrodynamic step in Sec. 6.1).  The transition column N_trans is the total H
column (HI + H2) from the surface at which 2 x_H2 first reaches 1/2 (Eq. e:NH_trans),
interpolated linearly between cell centres.

Readings: sigma_d,PE = 1e-21 Z'_d, sigma_d,LW = 1.5e-21 Z'_d; f_shld,C = 1 (TH85 is not
printed); N_eff is the column to the cell centre ("the perpendicular column", Sec. 7.2).
"""
from __future__ import annotations

import numpy as np

from . import YEAR_S, Params, default_params, step

N0_CR = 9.35e20
SIGMA_PE = 1.0e-21
SIGMA_LW = 1.5e-21


def f_shld_h2(N_h2, b5: float = 3.0):
    """Eq. e:fshld_H2_DB with x = N_H2 / 5e14 cm^-2."""
    x = np.asarray(N_h2, dtype=np.float64) / 5e14
    s = np.sqrt(1.0 + x)
    return 0.965 / (1.0 + x / b5) ** 2 + 0.035 / s * np.exp(-8.5e-4 * s)


def cell_average(t):
    t = np.asarray(t, dtype=np.float64)
    safe = np.where(t < 1e-8, 1.0, t)
    return np.where(t < 1e-8, 1.0 - 0.5 * t, -np.expm1(-safe) / safe)


def beamed_fields(n, xH2, dx, chi0, xi0, Zd):
    """chi_PE, chi_LW, f_shld,H2, xi and the centre columns N_c of one slab (arrays over
    its cells, cell 0 at the surface)."""
    n = np.asarray(n, dtype=np.float64)
    q = n * dx
    qh = (xH2 * n) * dx
    N_in = np.concatenate(([0.0], np.cumsum(q)[:-1]))     # column in front of the cell
    H_in = np.concatenate(([0.0], np.cumsum(qh)[:-1]))
    sp, sl = SIGMA_PE * Zd, SIGMA_LW * Zd
    chi_pe = chi0 * np.exp(-sp * N_in) * cell_average(sp * q)
    chi_lw = chi0 * np.exp(-sl * N_in) * cell_average(sl * q)
    f_h2 = f_shld_h2(H_in + 0.5 * xH2 * n * dx)
    N_c = N_in + 0.5 * q
    xi = np.where(N_c <= N0_CR, xi0, xi0 * N0_CR / np.maximum(N_c, N0_CR))
    return chi_pe, chi_lw, f_h2, xi, N_c


def transition_column(N_c, xH2):
    """Total H column at which 2 x_H2 first reaches 0.5, linear between cell centres
    (N_c[0] if the first cell is already past it; -1 if no cell reaches it)."""
    y = 2.0 * np.asarray(xH2)
    for i in range(y.size):
        if y[i] >= 0.5:
            if i == 0:
                return float(N_c[0])
            w = (0.5 - y[i - 1]) / (y[i] - y[i - 1])
            return float(N_c[i - 1] + w * (N_c[i] - N_c[i - 1]))
    return -1.0


def slabs(n, chi0, xi0, Z, dx, ncell: int, params: Params | None = None, t_end: float = 3e2 * 1e6 * YEAR_S,
          nchunk: int = 300, T_init: float = 100.0, xH2_init: float = 0.0, xHp_init: float = 1e-4) -> dict:
    """Evolves one slab per entry of the per-slab arrays n, chi0, xi0, Z (= Z'_g = Z'_d),
    dx.  Returns arrays [nslab, ncell] of T, xH2, xHp, xe, xCO, chi_pe, f_h2, N_c and
    status (OR over chunks), and N_trans [nslab]."""
    base = params if params is not None else default_params(mode=1)
    n, chi0, xi0, Z, dx = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (n, chi0, xi0, Z, dx))
    ns = n.size
    out = {k: np.zeros((ns, ncell)) for k in ("T", "xH2", "xHp", "xe", "xCO", "chi_pe", "f_h2", "N_c")}
    out["status"] = np.zeros((ns, ncell), dtype=np.int32)
    out["N_trans"] = np.zeros(ns)
    dt = t_end / nchunk
    for s in range(ns):
        p = Params.from_buffer_copy(base)
        p.chi0 = chi0[s]
        nn = np.full(ncell, n[s])
        T = np.full(ncell, T_init)
        x2 = np.full(ncell, xH2_init)
        xp = np.full(ncell, xHp_init)
        st = np.zeros(ncell, dtype=np.int32)
        r = None
        for k in range(nchunk):
            chi_pe, chi_lw, f_h2, xi, N_c = beamed_fields(nn, x2, dx[s], chi0[s], xi0[s], Z[s])
            cells = dict(n=nn, chi_pe=chi_pe, chi_lw=chi_lw, f_h2=f_h2, f_c=1.0, F_lyc=0.0, xi=xi, Zg=Z[s], Zd=Z[s],
                         T=T, xH2=x2, xHp=xp)
            r = step(cells, dt, p)
            T, x2, xp = r["T"], r["xH2"], r["xHp"]
            st |= r["status"]
        chi_pe, chi_lw, f_h2, xi, N_c = beamed_fields(nn, x2, dx[s], chi0[s], xi0[s], Z[s])
        out["T"][s], out["xH2"][s], out["xHp"][s] = T, x2, xp
        out["xe"][s], out["xCO"][s] = r["xe"], r["xCO"]
        out["chi_pe"][s], out["f_h2"][s], out["N_c"][s] = chi_pe, f_h2, N_c
        out["status"][s] = st
        out["N_trans"][s] = transition_column(N_c, x2)
    return out


def bialy_sternberg_ntrans(chi0, n, k_gr: float = 3e-17, sigma_tilde: float = 1.0, beta: float = 0.7):
    """The analytic transition column the paper quotes (Eqs. e:alpha, e:G, e:NH_trans)."""
    alpha = 3.8e4 * chi0 * (3.0e-17 / k_gr) * (1e2 / n)
    G = 3.0e-5 * sigma_tilde * (9.9 / (1.0 + 8.9 * sigma_tilde)) ** 0.37
    sigma_d = 1.9e-21 * sigma_tilde
    return beta / sigma_d * np.log(1.0 + (alpha * G / 2.0) ** (1.0 / beta))
