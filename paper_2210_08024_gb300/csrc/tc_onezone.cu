// One-zone equilibrium-curve driver kernels (Sec. 7.1; include/tc_onezone.h).
//
// These are bandwidth-trivial helpers around the step launches: a few dozen bytes per
// cell per chunk, against the thousands of FP64 operations the step does per cell.
#include <math.h>

#include "tc_onezone.cuh"

namespace tcg {

namespace {

constexpr double N0_CRATT = 9.35e20;   // Eq. e:cratt
constexpr double SIG_PE = 1.0e-21;     // sigma_d,PE per Z'_d (Sec. 5.3)
constexpr double SIG_LW = 1.5e-21;     // sigma_d,LW per Z'_d (Sec. 2.4, absorption)

// Eq. e:fshld_H2_DB with b_5 = 3 and x = N_H2 / 5e14 cm^-2.
__device__ __forceinline__ double f_shld_db(double N_h2) {
  const double x = N_h2 / 5e14;
  const double s = sqrt(1.0 + x);
  const double q = 1.0 + x / 3.0;
  return 0.965 / (q * q) + 0.035 / s * exp(-8.5e-4 * s);
}

__global__ void k_eq_fields(EqGrid g, EqWork w, double* __restrict__ T, double* __restrict__ xH2,
                            double* __restrict__ xHp, int chunk, int last) {
  const long long ncell = g.nn * (long long)g.ncurve;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / g.nn);
    const double n = g.n_axis[i - (long long)c * g.nn];
    const double chi0 = g.chi0[c], xi0 = g.xi0[c], Zd = g.Zd[c];
    if (chunk == 0) {
      T[i] = g.T0;
      xH2[i] = g.xH20;
      xHp[i] = g.xHp0;
      w.st_acc[i] = 0;
      w.n[i] = n;
      w.Zg[i] = g.Zg[c];
      w.Zd[i] = Zd;
      w.chi0[i] = chi0;
      if (!g.shielded) {
        w.chi_pe[i] = chi0;
        w.chi_lw[i] = chi0;
        w.fh2[i] = 1.0;
        w.xi[i] = xi0;
      }
    } else {
      w.st_acc[i] |= w.st[i];
    }
    if (g.shielded) {
      // Sec. 7.1.2: shielding length, column, attenuated fields and H2 self-shielding
      const double L = g.L0_cm * pow(n / g.n0, -g.a);
      const double N = n * L;
      w.chi_pe[i] = chi0 * exp(-SIG_PE * Zd * N);
      w.chi_lw[i] = chi0 * exp(-SIG_LW * Zd * N);
      w.xi[i] = (N <= N0_CRATT) ? xi0 : xi0 * N0_CRATT / N;
      w.fh2[i] = f_shld_db(0.5 * xH2[i] * n * L);
    }
    if (last) {
      w.prev[i] = T[i];
      w.prev[ncell + i] = xH2[i];
      w.prev[2 * ncell + i] = xHp[i];
    }
  }
}

__global__ void k_eq_finish(EqGrid g, EqWork w, const double* __restrict__ T, const double* __restrict__ xH2,
                            const double* __restrict__ xHp, const double* __restrict__ xe, double* __restrict__ P,
                            double* __restrict__ chg, int* __restrict__ status) {
  const long long ncell = g.nn * (long long)g.ncurve;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    const double n = g.n_axis[i % g.nn];
    P[i] = (1.1 + xe[i] - xH2[i]) * n * T[i];
    if (chg) {
      const double Tp = w.prev[i];
      const double d2 = fabs(xH2[i] - w.prev[ncell + i]);
      const double dp = fabs(xHp[i] - w.prev[2 * ncell + i]);
      chg[i] = fmax(fabs(T[i] - Tp) / Tp, fmax(d2, dp));
    }
    if (status) status[i] = w.st_acc[i] | w.st[i];
  }
}

// One thread per curve: a sequential scan of nn pressures (nn is at most thousands).
__global__ void k_eq_extrema(EqGrid g, const double* __restrict__ P, int* __restrict__ i_max,
                             int* __restrict__ i_min) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncurve) return;
  const double* p = P + (long long)c * g.nn;
  long long imax = -1, imin = -1;
  for (long long i = 0; i + 1 < g.nn; ++i)
    if (p[i + 1] < p[i]) { imax = i; break; }
  if (imax >= 0)
    for (long long j = imax; j + 1 < g.nn; ++j)
      if (p[j + 1] > p[j]) { imin = j; break; }
  if (i_max) i_max[c] = (int)imax;
  if (i_min) i_min[c] = (int)imin;
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_eq_fields(const EqGrid& g, const EqWork& w, double* T, double* xH2, double* xHp, int chunk,
                             bool last, cudaStream_t st) {
  k_eq_fields<<<grid_for(g.nn * g.ncurve), 256, 0, st>>>(g, w, T, xH2, xHp, chunk, last ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_eq_finish(const EqGrid& g, const EqWork& w, const double* T, const double* xH2,
                             const double* xHp, const double* xe, double* P, double* chg, int* status,
                             cudaStream_t st) {
  k_eq_finish<<<grid_for(g.nn * g.ncurve), 256, 0, st>>>(g, w, T, xH2, xHp, xe, P, chg, status);
  return cudaGetLastError();
}

cudaError_t launch_eq_extrema(const EqGrid& g, const double* P, int* i_max, int* i_min, cudaStream_t st) {
  k_eq_extrema<<<(g.ncurve + 63) / 64, 64, 0, st>>>(g, P, i_max, i_min);
  return cudaGetLastError();
}

}  // namespace tcg
