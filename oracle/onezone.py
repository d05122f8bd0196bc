"""One-zone thermal-equilibrium curves (Sec. 7.1), oracle side.

TEST INFRASTRUCTURE ONLY: the plain statement of the one-zone driver that the CUDA
library runs on the GPU (tc_eq_curves).  Only tests/ and bench.py's CPU legs may call
it; it shares no code with the library.

Sec. 7.1: a cell of given n_H, FUV intensity, CR rate and abundances is evolved at
fixed density for ~1e2 Myr until temperature and abundances settle; the thermal
pressure P/k_B = (1.1 + x_e - x_H2) n_H T of the settled state, over a grid of
densities, traces the equilibrium curve of Figs. f:equil_unshld and f:equil_shld.

* Unshielded (Sec. 7.1.1): chi_PE = chi_LW = chi0, no H2 or C shielding, xi = xi0.
* Shielded (Sec. 7.1.2): a shielding length L = L0 (n_H/n0)^-a (L0 = 5 pc, n0 = 1e2,
  a = 0.7) and column N = n_H L give chi_PE/LW = chi0 exp(-sigma_d,PE/LW N), the CR
  rate of Eq. e:cratt with N_eff = N, and the H2 self-shielding factor of
  Eq. e:fshld_H2_DB at N_H2 = 0.5 n_H2 L from the current H2 abundance.

Readings (the paper is silent):
* The ~1e2 Myr is integrated in `nchunk` equal chunks.  Between chunks the shielded
  fields are recomputed from the current x_H2 and held fixed over the next chunk, as
  the radiation is held fixed over a hydrodynamic step (Sec. 6.1).  The change of the
  state over the last chunk is reported as the steady-state residual.
* C shielding (TH85) is not printed: f_shld,C = 1.
* sigma_d,PE = 1e-21 Z'_d (Sec. 5.3) and sigma_d,LW = 1.5e-21 Z'_d (Sec. 2.4, absorption).
* P_max is taken at the first density where P falls to the next grid point, P_min at
  the first density at or after it where P rises to the next grid point.
"""
from __future__ import annotations

import numpy as np

from . import YEAR_S, Params, default_params, step

PC_CM = 3.0856775814913673e18
MYR_S = 1e6 * YEAR_S
N0_CR = 9.35e20          # Eq. e:cratt
SIGMA_PE = 1.0e-21       # per Z'_d, Sec. 5.3
SIGMA_LW = 1.5e-21       # per Z'_d, Sec. 2.4 (absorption)


def f_shld_h2(N_h2, b5: float = 3.0):
    """Draine & Bertoldi H2 self-shielding, Eq. e:fshld_H2_DB, x = N_H2 / 5e14 cm^-2."""
    x = np.asarray(N_h2, dtype=np.float64) / 5e14
    s = np.sqrt(1.0 + x)
    return 0.965 / (1.0 + x / b5) ** 2 + 0.035 / s * np.exp(-8.5e-4 * s)


def xi_attenuated(xi0, N_eff):
    """Eq. e:cratt: xi0 up to N_0, then xi0 (N_eff/N_0)^-1."""
    N_eff = np.asarray(N_eff, dtype=np.float64)
    return np.where(N_eff <= N0_CR, xi0, xi0 * N0_CR / np.maximum(N_eff, N0_CR))


def shielding_length_cm(n, L0_pc: float = 5.0, n0: float = 1e2, a: float = 0.7):
    """Sec. 7.1.2: L_shld = L0 (n_H / n0)^-a."""
    return L0_pc * PC_CM * (np.asarray(n, dtype=np.float64) / n0) ** (-a)


def shielded_fields(n, xH2, chi0, xi0, Zd, L0_pc=5.0, n0=1e2, a=0.7):
    """chi_PE, chi_LW, f_shld,H2 and xi of the Sec. 7.1.2 prescription."""
    L = shielding_length_cm(n, L0_pc, n0, a)
    N = np.asarray(n) * L
    chi_pe = chi0 * np.exp(-SIGMA_PE * Zd * N)
    chi_lw = chi0 * np.exp(-SIGMA_LW * Zd * N)
    f_h2 = f_shld_h2(0.5 * np.asarray(xH2) * np.asarray(n) * L)
    return chi_pe, chi_lw, f_h2, xi_attenuated(xi0, N)


def pressure_k(n, T, xe, xH2):
    """P / k_B = n_tot T with n_tot = (1.1 + x_e - x_H2) n_H (He at 0.1 per H)."""
    return (1.1 + xe - xH2) * n * T


def extrema(P):
    """(i_max, i_min) of one curve: i_max is the first index whose pressure exceeds the
    next one's (the end of the warm branch), i_min the first index at or after i_max whose
    pressure is below the next one's (the start of the cold branch).  -1 where absent."""
    P = np.asarray(P)
    imax = imin = -1
    for i in range(P.size - 1):
        if P[i + 1] < P[i]:
            imax = i
            break
    if imax >= 0:
        for j in range(imax, P.size - 1):
            if P[j + 1] > P[j]:
                imin = j
                break
    return imax, imin


def curves(n_axis, chi0, xi0, Zg, Zd, params: Params | None = None, t_end: float = 1e2 * MYR_S,
           nchunk: int = 10, shielded: bool = False, L0_pc: float = 5.0, n0: float = 1e2, a: float = 0.7,
           T_init: float = 3000.0, xH2_init: float = 0.0, xHp_init: float = 1e-2) -> dict:
    """Equilibrium curves over the density axis `n_axis` for each curve c with
    (chi0[c], xi0[c], Zg[c], Zd[c]).  Returns arrays of shape (ncurve, nn): T, xH2, xHp,
    xe, xCO, P (P/k_B), chg (largest change over the last chunk: relative for T, absolute
    for the abundances) and status (OR over chunks); and i_max, i_min per curve."""
    base = params if params is not None else default_params(mode=1)
    n = np.asarray(n_axis, dtype=np.float64)
    nn = n.size
    chi0, xi0, Zg, Zd = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (chi0, xi0, Zg, Zd))
    nc = chi0.size
    keys = ("T", "xH2", "xHp", "xe", "xCO", "P", "chg")
    out = {k: np.zeros((nc, nn)) for k in keys}
    out["status"] = np.zeros((nc, nn), dtype=np.int32)
    out["i_max"] = np.full(nc, -1, dtype=np.int32)
    out["i_min"] = np.full(nc, -1, dtype=np.int32)
    dt = t_end / nchunk
    for c in range(nc):
        p = Params.from_buffer_copy(base)
        p.chi0 = chi0[c]       # unattenuated FUV scale of the optical dust heating (Sec. 4.3.6)
        T = np.full(nn, T_init)
        x2 = np.full(nn, xH2_init)
        xp = np.full(nn, xHp_init)
        st = np.zeros(nn, dtype=np.int32)
        prev = None
        r = None
        for k in range(nchunk):
            if shielded:
                chi_pe, chi_lw, f_h2, xi = shielded_fields(n, x2, chi0[c], xi0[c], Zd[c], L0_pc, n0, a)
            else:
                chi_pe, chi_lw, f_h2, xi = chi0[c], chi0[c], 1.0, xi0[c]
            if k == nchunk - 1:
                prev = (T.copy(), x2.copy(), xp.copy())
            cells = dict(n=n, chi_pe=chi_pe, chi_lw=chi_lw, f_h2=f_h2, f_c=1.0, F_lyc=0.0, xi=xi,
                         Zg=Zg[c], Zd=Zd[c], T=T, xH2=x2, xHp=xp)
            r = step(cells, dt, p)
            T, x2, xp = r["T"], r["xH2"], r["xHp"]
            st |= r["status"]
        out["T"][c], out["xH2"][c], out["xHp"][c] = T, x2, xp
        out["xe"][c], out["xCO"][c] = r["xe"], r["xCO"]
        out["status"][c] = st
        out["P"][c] = pressure_k(n, T, r["xe"], x2)
        out["chg"][c] = np.maximum(np.abs(T - prev[0]) / prev[0], np.maximum(np.abs(x2 - prev[1]), np.abs(xp - prev[2])))
        out["i_max"][c], out["i_min"][c] = extrema(out["P"][c])
    return out
