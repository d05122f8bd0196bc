// Device side of the one-zone equilibrium-curve driver (include/tc_onezone.h):
// per-chunk field set-up, the end-of-run pressure and residual, and the per-curve
// extrema.  The step itself is the library's persistent step kernel.
#pragma once
#include <cuda_runtime.h>

namespace tcg {

// Per-cell workspace of the driver (device arrays of length ncell = ncurve * nn).
struct EqWork {
  double *n, *chi_pe, *chi_lw, *fh2, *xi, *Zg, *Zd, *chi0;  // step inputs
  double *prev;       // [3][ncell]: T, x_H2, x_H+ before the last chunk
  int *st, *st_acc;   // status of the latest launch; OR over the earlier ones
};

// The grid: curve parameters (device copies, [ncurve]) and the shielding prescription.
struct EqGrid {
  const double* n_axis;  // [nn]
  const double *chi0, *xi0, *Zg, *Zd;
  long long nn;
  int ncurve;
  int shielded;
  double L0_cm, n0, a;   // Sec. 7.1.2: L = L0 (n/n0)^-a
  double T0, xH20, xHp0;
};

// Chunk set-up: on chunk 0 the start state and the fixed inputs; on later chunks the
// previous launch's status is OR-ed into st_acc; shielded fields are recomputed from
// the current x_H2 every chunk; before the last chunk the state is saved to prev.
cudaError_t launch_eq_fields(const EqGrid& g, const EqWork& w, double* T, double* xH2, double* xHp, int chunk,
                             bool last, cudaStream_t st);
// P/k_B, the last-chunk change and the OR of all statuses (chg and status may be null).
cudaError_t launch_eq_finish(const EqGrid& g, const EqWork& w, const double* T, const double* xH2,
                             const double* xHp, const double* xe, double* P, double* chg, int* status,
                             cudaStream_t st);
// Per-curve extrema of P (i_max, i_min may be null).
cudaError_t launch_eq_extrema(const EqGrid& g, const double* P, int* i_max, int* i_min, cudaStream_t st);

}  // namespace tcg
