/*
 * tc_pdr.h -- plane-parallel PDR slabs and the HI-to-H2 transition column on the GPU.
 *
 * Kim, Gong, Kim & Ostriker (2023, arXiv:2210.08024), Secs. 7.2 and 7.3: a uniform
 * slab lit from one face by a beamed FUV field at normal incidence, evolved until
 * temperature, abundances and shielding settle.  Sec. 7.3 compares the total H column
 * at which 2 x_H2 reaches 1/2 with the analytic approximation of Eq. e:NH_trans.
 *
 * A cell behind the column N = sum of n_H dx over the cells in front of it (cell 0 is
 * at the lit surface) sees, averaged over the cell (Eq. e:Erad with one ray),
 *   chi_j = chi0 exp(-sigma_j N) g(sigma_j n_H dx),  g(t) = (1 - e^-t)/t,  j = PE, LW,
 * with sigma_d,PE = 1e-21 Z'_d and sigma_d,LW = 1.5e-21 Z'_d.  It also sees the H2
 * self-shielding factor of Eq. e:fshld_H2_DB (b_5 = 3) at the H2 column to its centre,
 * and the CR rate of Eq. e:cratt with N_eff the column to its centre ("the
 * perpendicular column").  C shielding is not modelled (f_shld,C = 1).  The time t_end
 * is split into nchunk equal chunks; before each chunk the fields are recomputed from
 * the current x_H2 (one warp scans each slab), then one persistent step launch advances
 * every cell of every slab with the handle's tc_params.
 */
#ifndef TC_PDR_H
#define TC_PDR_H

#include "tc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_pdr_spec {
  const double *n;      /* HOST [nslab]: n_H of each slab [cm^-3], > 0 */
  const double *chi0;   /* HOST [nslab]: beamed FUV intensity at the surface (Draine units), >= 0 */
  const double *xi0;    /* HOST [nslab]: unattenuated CR ionisation rate [s^-1], >= 0 */
  const double *Z;      /* HOST [nslab]: Z'_g = Z'_d, >= 0 */
  const double *dx_cm;  /* HOST [nslab]: cell size [cm], > 0 */
  int nslab;            /* >= 1 */
  long long ncell;      /* cells per slab, >= 1 */
  double t_end_s;       /* total time [s] (3e2 Myr) */
  int nchunk;           /* >= 1 (300) */
  double T_init, xH2_init, xHp_init;  /* start state (100 K, 0, 1e-4) */
} tc_pdr_spec;

/* DEVICE outputs, slab-major: element [s * ncell + i] is cell i of slab s. */
typedef struct tc_pdr_out {
  double *T, *x_h2, *x_hp, *x_e;   /* required: the state after t_end */
  double *x_co;                    /* optional */
  double *chi_pe, *f_shld_h2;      /* optional: the fields of the final state */
  double *N_c;                     /* optional: total H column from the surface to each cell centre */
  int *status;                     /* optional: TC_ST_* bits OR-ed over all chunks */
  double *N_trans;                 /* optional [nslab]: H column where 2 x_H2 first reaches 1/2,
                                      linear between cell centres; -1 if never */
} tc_pdr_out;

/* Defaults: t_end = 3e2 Myr in 300 chunks, start state 100 K, x_H2 = 0, x_H+ = 1e-4. */
int tc_pdr_spec_default(tc_pdr_spec *s);

/* Waits for the work already on `stream`, copies the host arrays of `s`, then enqueues
 * the run (per chunk: a field kernel and a step launch; then the final fields and the
 * transition columns) and returns without waiting for it.  Shares the handle's driver
 * workspace with tc_eq_curves (11 doubles and 3 ints per cell, grown by cudaMalloc).
 * TC_EINVAL for a bad spec or output, TC_ENOMLP for a seeded mode without weights. */
int tc_pdr(tc_handle *h, const tc_pdr_spec *s, const tc_pdr_out *o, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TC_PDR_H */
