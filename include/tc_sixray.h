/*
 * tc_sixray.h -- six-ray FUV fields, H2 self-shielding and CR attenuation on a uniform
 * Cartesian grid, on the GPU.
 *
 * Kim, Gong, Kim & Ostriker (2023, arXiv:2210.08024), Sec. 5.2: rays enter through the
 * six faces of the domain along +-x, +-y and +-z, each carrying one sixth of the
 * isotropic unattenuated field chi0, and are attenuated by dust.  For band j (PE, LW)
 * with dust cross section sigma_j per H, the field a ray leaves in a cell, averaged
 * over the cell (Eq. e:Erad with Delta s = dx), is exp(-sigma_j N) g(sigma_j n_H dx)
 * times its entering value, N the column n_H dx summed over the cells between the face
 * and the cell and g(t) = (1 - e^-t)/t.  So
 *
 *   chi_j = (chi0/6) sum_rays exp(-sigma_j N_ray) g(sigma_j n_H dx),   j = PE, LW.
 *
 * Eq. e:Erad_H2 weights each LW ray by the H2 self-shielding factor of Eq. e:fshld_H2_DB
 * (b_5 = 3) at the ray's H2 column to the cell centre (N_H2,ray + 0.5 x_H2 n_H dx):
 * f_shld,H2 = sum_rays w f / sum_rays w with w = exp(-sigma_LW N_ray), so that
 * chi_H2 = chi_LW f_shld,H2 (Eq. e:chi_H2).  Sec. 5.3: N_eff = -ln(chi_PE/chi0)/sigma_d,PE
 * (Eq. e:tau_eff) and xi = xi0 min(1, N_0/N_eff) with N_0 = 9.35e20 cm^-2 (Eq. e:cratt).
 *
 * sigma_d,PE = 1e-21 Z'_d and sigma_d,LW = 1.5e-21 Z'_d cm^2 per H (Sec. 5.3; Sec. 2.4,
 * absorption); Z'_d is uniform.  Sums over rays are formed relative to the smallest
 * column, so cells whose fields underflow still get a finite f_shld,H2 and N_eff.  With
 * Z'_d = 0 there is no dust column: N_eff = 0 and xi = xi0.  The C shielding factor
 * (TH85, not printed in the paper) is not computed.
 *
 * Outputs are the step's radiation inputs (tc_fields.chi_pe, chi_lw, f_shld_h2, xi_cr).
 */
#ifndef TC_SIXRAY_H
#define TC_SIXRAY_H

#include "tc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_sixray_grid {
  long long nx, ny, nz;  /* cells per axis, each >= 1; cell (i, j, k) is element i + nx (j + ny k) */
  double dx_cm;          /* cell size [cm], > 0 */
  double chi0;           /* unattenuated isotropic FUV intensity at the faces (Draine units), >= 0 */
  double xi0;            /* unattenuated CR ionisation rate per H [s^-1], >= 0 */
  double Zd;             /* dust abundance relative to solar, >= 0, uniform */
} tc_sixray_grid;

/* n (n_H [cm^-3]) and x_h2 are caller-owned DEVICE arrays of nx*ny*nz doubles; chi_pe,
 * chi_lw, f_shld_h2 and xi_cr are DEVICE outputs of the same length (8-byte aligned),
 * N_eff an optional one (NULL to skip).  The outputs double as the workspace of the
 * three axis passes (three kernel launches): the call allocates nothing.  Stream-ordered,
 * returns without synchronising.  TC_EINVAL for a bad grid or pointer. */
int tc_sixray(const tc_sixray_grid *g, const double *n, const double *x_h2, double *chi_pe, double *chi_lw,
              double *f_shld_h2, double *xi_cr, double *N_eff, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TC_SIXRAY_H */
