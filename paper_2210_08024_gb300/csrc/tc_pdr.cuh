// Device side of the PDR slab driver (include/tc_pdr.h).
#pragma once
#include <cuda_runtime.h>

namespace tcg {

// Per-slab parameters (device copies, [nslab]) and the start state.
struct PdrSlabs {
  const double *n, *chi0, *xi0, *Z, *dx;
  int nslab;
  long long ncell;
  double T0, xH20, xHp0;
};

// Per-cell workspace (length nslab * ncell): step inputs and statuses.
struct PdrWork {
  double *n, *chi_pe, *chi_lw, *fh2, *xi, *Zg, *Zd, *chi0;
  int *st, *st_acc;
};

cudaError_t launch_pdr_fields(const PdrSlabs& g, const PdrWork& w, double* T, double* xH2, double* xHp, int chunk,
                              bool final_, double* out_chi_pe, double* out_fh2, double* out_Nc, cudaStream_t st);
// out[i] |= acc[i] over n elements.
cudaError_t launch_or_status(int* out, const int* acc, long long n, cudaStream_t st);
cudaError_t launch_pdr_ntrans(const PdrSlabs& g, const double* xH2, double* Ntr, cudaStream_t st);

}  // namespace tcg
