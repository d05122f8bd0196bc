"""Six-ray radiation fields and CR attenuation on a uniform Cartesian grid (Secs. 5.2,
5.3), oracle side.

TEST INFRASTRUCTURE ONLY: the plain statement of what the library's tc_sixray computes.
Only tests/ and bench.py's CPU legs may call it; it shares no code with the library.

Rays enter through the six faces of the domain along +-x, +-y, +-z, each carrying one
sixth of the isotropic unattenuated field chi0 (Sec. 5.2).  For band j (PE, LW) with
dust cross section sigma_j per H, a ray reaching a cell through a column N (n_H dx
summed over the cells between the face and the cell) deposits, averaged over the cell
(Eq. e:Erad with Delta s = dx),

    E_j,ray / E_j,0 = exp(-sigma_j N) g(sigma_j n_H dx),   g(t) = (1 - e^-t) / t,

so chi_j = (chi0 / 6) sum_rays exp(-sigma_j N_ray) g(sigma_j n_H dx).  The H2-dissociating
field (Eq. e:Erad_H2) weights each LW ray by the self-shielding factor of
Eq. e:fshld_H2_DB (b_5 = 3) at the ray's H2 column to the cell centre, N_H2,ray + 0.5
x_H2 n_H dx (the footnote to Eq. e:fshld_H2_DB), so f_shld,H2,eff = sum_rays w_ray f_ray /
sum_rays w_ray with w_ray = exp(-sigma_LW N_ray).  The effective column is
N_eff = tau_PE,eff / sigma_d,PE with tau_PE,eff = -ln(chi_PE / chi0) (Eq. e:tau_eff; the
unattenuated PE field is chi0), and xi follows Eq. e:cratt.

Readings: sigma_d,PE = 1e-21 Z'_d (Sec. 5.3), sigma_d,LW = 1.5e-21 Z'_d (Sec. 2.4,
absorption); Z'_d is uniform over the grid.  Sums over rays are taken relative to the
smallest column, so deep cells whose fields underflow still get a finite
f_shld,H2,eff and N_eff.  With Z'_d = 0 there is no dust column and xi = xi0.
The C shielding factor (TH85, not printed) is not computed.
"""
from __future__ import annotations

import numpy as np

N0_CR = 9.35e20          # Eq. e:cratt
SIGMA_PE = 1.0e-21       # per Z'_d
SIGMA_LW = 1.5e-21       # per Z'_d


def f_shld_h2(N_h2, b5: float = 3.0):
    """Eq. e:fshld_H2_DB with x = N_H2 / 5e14 cm^-2."""
    x = np.asarray(N_h2, dtype=np.float64) / 5e14
    s = np.sqrt(1.0 + x)
    return 0.965 / (1.0 + x / b5) ** 2 + 0.035 / s * np.exp(-8.5e-4 * s)


def cell_average(t):
    """g(t) = (1 - e^-t)/t, the mean of e^-s over a cell of optical depth t (1 - t/2 below 1e-8)."""
    t = np.asarray(t, dtype=np.float64)
    safe = np.where(t < 1e-8, 1.0, t)
    return np.where(t < 1e-8, 1.0 - 0.5 * t, -np.expm1(-safe) / safe)


def exclusive_cumsum(a, axis):
    """Sum of the elements before each one along `axis`, accumulated from the start."""
    c = np.cumsum(a, axis=axis)
    out = np.zeros_like(a)
    dst = [slice(None)] * a.ndim
    src = [slice(None)] * a.ndim
    dst[axis] = slice(1, None)
    src[axis] = slice(None, -1)
    out[tuple(dst)] = c[tuple(src)]
    return out


def ray_columns(q, dx):
    """Columns of q*dx from each of the six faces to each cell's near face, each
    accumulated from its ray's entry face (Sec. 5.2: optical depths are integrated from
    the domain boundary): a list of six arrays (rays along +x, -x, +y, -y, +z, -z),
    arrays indexed [z, y, x]."""
    out = []
    qd = q * dx
    for axis in (2, 1, 0):
        fwd = exclusive_cumsum(qd, axis)
        bwd = np.flip(exclusive_cumsum(np.flip(qd, axis), axis), axis)
        out += [fwd, bwd]
    return out


def sixray(n, xH2, dx, chi0=1.0, xi0=2e-16, Zd=1.0) -> dict:
    """n, xH2: arrays [nz, ny, nx]; dx in cm.  Returns chi_pe, chi_lw, f_h2, xi and N_eff."""
    n = np.asarray(n, dtype=np.float64)
    xH2 = np.asarray(xH2, dtype=np.float64)
    N = ray_columns(n, dx)
    NH2 = ray_columns(xH2 * n, dx)
    sp, sl = SIGMA_PE * Zd, SIGMA_LW * Zd
    Nmin = np.minimum.reduce(N)
    wpe = [np.exp(-sp * (Nr - Nmin)) for Nr in N]
    wlw = [np.exp(-sl * (Nr - Nmin)) for Nr in N]
    f = [f_shld_h2(Hr + 0.5 * xH2 * n * dx) for Hr in NH2]
    Spe = sum(wpe)
    Slw = sum(wlw)
    Sh2 = sum(w * fr for w, fr in zip(wlw, f))
    gpe = cell_average(sp * n * dx)
    glw = cell_average(sl * n * dx)
    chi_pe = chi0 / 6.0 * np.exp(-sp * Nmin) * Spe * gpe
    chi_lw = chi0 / 6.0 * np.exp(-sl * Nmin) * Slw * glw
    f_h2 = Sh2 / Slw
    if sp > 0.0:
        tau_eff = sp * Nmin - np.log(Spe * gpe / 6.0)
        N_eff = tau_eff / sp
    else:
        N_eff = np.zeros_like(n)
    xi = np.where(N_eff <= N0_CR, xi0, xi0 * N0_CR / np.maximum(N_eff, N0_CR))
    return dict(chi_pe=chi_pe, chi_lw=chi_lw, f_h2=f_h2, xi=xi, N_eff=N_eff)
