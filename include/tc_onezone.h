/*
 * tc_onezone.h -- one-zone thermal-equilibrium curves on the GPU.
 *
 * Sec. 7.1 of Kim, Gong, Kim & Ostriker (2023, arXiv:2210.08024) characterises the
 * model by cells held at fixed density, FUV intensity, CR rate and abundances and
 * evolved for ~1e2 Myr until temperature and abundances stop changing.  The settled
 * thermal pressure P/k_B = (1.1 + x_e - x_H2) n_H T over a range of n_H traces the
 * equilibrium curve (Figs. f:equil_unshld, f:equil_shld); its local maximum P_max (end
 * of the warm branch) and the following local minimum P_min (start of the cold branch)
 * bound the pressures at which warm and cold gas coexist (Fig. f:minmax).
 *
 * tc_eq_curves runs every (curve, density) cell of such a grid in one persistent step
 * launch per chunk of the integration, using the handle's tc_params (mode, flags,
 * dust-heating parameters, tolerances), and reduces the curves' extrema on the device.
 *
 *  - Unshielded (Sec. 7.1.1): chi_PE = chi_LW = chi0, f_shld,H2 = f_shld,C = 1, xi = xi0.
 *  - Shielded (Sec. 7.1.2): L = L0 (n_H/n0)^-a, N = n_H L, chi_PE/LW = chi0
 *    exp(-sigma_d,PE/LW N) with sigma_d,PE = 1e-21 Z'_d and sigma_d,LW = 1.5e-21 Z'_d,
 *    xi from Eq. e:cratt with N_eff = N, and f_shld,H2 from Eq. e:fshld_H2_DB (b_5 = 3)
 *    at N_H2 = 0.5 x_H2 n_H L.  C shielding is not modelled (f_shld,C = 1).  The fields are
 *    recomputed from the current x_H2 before each chunk and held over it.
 *  - The optical dust heating of each curve scales with its own chi0 (Sec. 4.3.6); the
 *    handle's T_cmb, opt_over_fuv and tau_opt_over_tau_pe apply to all curves (Sec. 7.1.2
 *    uses T_rad = 6 K and tau_OPT = tau_PE / 1.87).
 */
#ifndef TC_ONEZONE_H
#define TC_ONEZONE_H

#include "tc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_eq_spec {
  const double *n_axis;     /* HOST, nn densities n_H [cm^-3] shared by every curve, each > 0 */
  long long nn;             /* densities per curve, >= 1 */
  const double *chi0;       /* HOST, ncurve unattenuated FUV intensities (Draine units), >= 0 */
  const double *xi0;        /* HOST, ncurve unattenuated CR ionisation rates per H [s^-1], >= 0 */
  const double *Zg, *Zd;    /* HOST, ncurve gas-metal and dust abundances relative to solar, >= 0 */
  int ncurve;               /* >= 1 */
  int shielded;             /* 0: Sec. 7.1.1 (unshielded); 1: Sec. 7.1.2 prescription */
  double L_shld0_pc;        /* Sec. 7.1.2 shielding length at n0 [pc] (5) */
  double n_shld0;           /* Sec. 7.1.2 reference density [cm^-3] (1e2) */
  double a_shld;            /* Sec. 7.1.2 power-law index (0.7) */
  double t_end_s;           /* total time [s] (Sec. 7.1: ~1e2 Myr) */
  int nchunk;               /* equal chunks the time is split into, >= 1 */
  double T_init, xH2_init, xHp_init;  /* start state of every cell (3000 K, 0, 1e-2) */
} tc_eq_spec;

/* Output arrays: caller-owned DEVICE pointers, 8-byte aligned, curve-major: element
 * [c * nn + i] belongs to curve c at n_axis[i]. */
typedef struct tc_eq_out {
  double *T, *x_h2, *x_hp;  /* required: the state after t_end */
  double *x_e;              /* required: electron abundance at that state */
  double *P_k;              /* required: P / k_B = (1.1 + x_e - x_H2) n_H T [K cm^-3] */
  double *x_co;             /* optional (NULL): CO abundance */
  double *chg;              /* optional: change over the last chunk, max(|dT|/T, |dx_H2|, |dx_H+|) */
  int *status;              /* optional: TC_ST_* bits OR-ed over all chunks */
  int *i_max, *i_min;       /* optional, [ncurve]: index of P_max = the first i with
                               P[i+1] < P[i], and of P_min = the first j >= i_max with
                               P[j+1] > P[j]; -1 where absent */
} tc_eq_out;

/* Defaults: unshielded, L0 = 5 pc, n0 = 1e2 cm^-3, a = 0.7, t_end = 1e2 Myr, 10 chunks,
 * start state 3000 K, x_H2 = 0, x_H+ = 1e-2.  The caller sets the axis and curve arrays. */
int tc_eq_spec_default(tc_eq_spec *s);

/* Waits for the work already on `stream`, copies the host arrays of `s` to the device,
 * then enqueues the whole integration (nchunk step launches, each preceded by a small
 * set-up kernel, and two reduction kernels) and returns without waiting for it.  The
 * handle keeps a device workspace of 11 doubles and 3 ints per cell, grown (cudaMalloc)
 * when a call needs more.  TC_EINVAL for a bad spec or output (non-finite or negative
 * values, n_H <= 0, 2 x_H2 + x_H+ > 1), TC_ENOMLP for a seeded mode without weights. */
int tc_eq_curves(tc_handle *h, const tc_eq_spec *s, const tc_eq_out *o, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TC_ONEZONE_H */
