// Plane-parallel PDR slab kernels (Secs. 7.2, 7.3; include/tc_pdr.h): the beamed
// fields of every slab (one warp per slab, the column in front of each cell by a
// chunked shuffle scan) and the transition columns.
#include <math.h>

#include "tc_pdr.cuh"

namespace tcg {
namespace {

constexpr double N0_CRATT = 9.35e20;  // Eq. e:cratt

__device__ __forceinline__ double f_shld_db(double N_h2) {  // Eq. e:fshld_H2_DB, b_5 = 3
  const double x = N_h2 / 5e14;
  const double s = sqrt(1.0 + x);
  const double q = 1.0 + x / 3.0;
  return 0.965 / (q * q) + 0.035 / s * exp(-8.5e-4 * s);
}

__device__ __forceinline__ double cell_average(double t) {  // (1 - e^-t)/t
  return (t < 1e-8) ? 1.0 - 0.5 * t : -expm1(-t) / t;
}

// One warp per slab.  chunk == 0: the start state and the fixed inputs; chunk > 0: the
// previous step's status is OR-ed into st_acc.  final: the fields of the final state go
// to the optional outputs instead of the step inputs.
__global__ void __launch_bounds__(256) k_pdr_fields(PdrSlabs g, PdrWork w, double* __restrict__ T,
                                                    double* __restrict__ xH2, double* __restrict__ xHp, int chunk,
                                                    int final_, double* __restrict__ out_chi_pe,
                                                    double* __restrict__ out_fh2, double* __restrict__ out_Nc) {
  const int slab = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (slab >= g.nslab) return;
  const double n = g.n[slab], dx = g.dx[slab], chi0 = g.chi0[slab], xi0 = g.xi0[slab], Z = g.Z[slab];
  const double spe = 1.0e-21 * Z, slw = 1.5e-21 * Z;
  const double q = n * dx;
  const double gpe = cell_average(spe * q), glw = cell_average(slw * q);
  const long long base = (long long)slab * g.ncell;
  double carryN = 0.0, carryH = 0.0;
  for (long long i0 = 0; i0 < g.ncell; i0 += 32) {
    const long long i = i0 + lane;
    const bool live = i < g.ncell;
    const long long e = base + i;
    if (live && chunk == 0 && !final_) {
      T[e] = g.T0;
      xH2[e] = g.xH20;
      xHp[e] = g.xHp0;
      w.st_acc[e] = 0;
      w.n[e] = n;
      w.Zg[e] = Z;
      w.Zd[e] = Z;
      w.chi0[e] = chi0;
    } else if (live && !final_) {
      w.st_acc[e] |= w.st[e];
    }
    const double x2 = live ? xH2[e] : 0.0;
    const double qh = (x2 * n) * dx;
    // column in front of the cell: exclusive scans of q (constant) and q_H2
    double iN = live ? q : 0.0, iH = qh;
    for (int d = 1; d < 32; d <<= 1) {
      const double vN = __shfl_up_sync(0xffffffffu, iN, d);
      const double vH = __shfl_up_sync(0xffffffffu, iH, d);
      if (lane >= d) { iN += vN; iH += vH; }
    }
    double eN = __shfl_up_sync(0xffffffffu, iN, 1), eH = __shfl_up_sync(0xffffffffu, iH, 1);
    if (lane == 0) { eN = 0.0; eH = 0.0; }
    const double totN = __shfl_sync(0xffffffffu, iN, 31), totH = __shfl_sync(0xffffffffu, iH, 31);
    if (live) {
      const double Nin = carryN + eN, Hin = carryH + eH;
      const double chi_pe = chi0 * exp(-spe * Nin) * gpe;
      const double fh2 = f_shld_db(Hin + 0.5 * x2 * n * dx);
      const double Nc = Nin + 0.5 * q;
      if (final_) {
        if (out_chi_pe) out_chi_pe[e] = chi_pe;
        if (out_fh2) out_fh2[e] = fh2;
        if (out_Nc) out_Nc[e] = Nc;
      } else {
        w.chi_pe[e] = chi_pe;
        w.chi_lw[e] = chi0 * exp(-slw * Nin) * glw;
        w.fh2[e] = fh2;
        w.xi[e] = (Nc <= N0_CRATT) ? xi0 : xi0 * N0_CRATT / Nc;
      }
    }
    carryN += totN;
    carryH += totH;
  }
}

// One thread per slab: the first cell with 2 x_H2 >= 1/2, interpolated in the column.
__global__ void k_pdr_ntrans(PdrSlabs g, const double* __restrict__ xH2, double* __restrict__ Ntr) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.nslab) return;
  const double q = g.n[s] * g.dx[s];
  const double* x = xH2 + (long long)s * g.ncell;
  double r = -1.0;
  double Nprev = 0.0, yprev = 0.0, Nin = 0.0;
  for (long long i = 0; i < g.ncell; ++i) {
    const double Nc = Nin + 0.5 * q;
    const double y = 2.0 * x[i];
    if (y >= 0.5) {
      r = (i == 0) ? Nc : Nprev + (0.5 - yprev) / (y - yprev) * (Nc - Nprev);
      break;
    }
    Nprev = Nc;
    yprev = y;
    Nin += q;
  }
  Ntr[s] = r;
}

__global__ void k_or_status(int* __restrict__ out, const int* __restrict__ acc, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] |= acc[i];
}

}  // namespace

cudaError_t launch_or_status(int* out, const int* acc, long long n, cudaStream_t st) {
  long long b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  k_or_status<<<(int)(b < 1 ? 1 : b), 256, 0, st>>>(out, acc, n);
  return cudaGetLastError();
}

cudaError_t launch_pdr_fields(const PdrSlabs& g, const PdrWork& w, double* T, double* xH2, double* xHp, int chunk,
                              bool final_, double* out_chi_pe, double* out_fh2, double* out_Nc, cudaStream_t st) {
  const int warps_per_block = 8;
  const int blocks = (g.nslab + warps_per_block - 1) / warps_per_block;
  k_pdr_fields<<<blocks, 32 * warps_per_block, 0, st>>>(g, w, T, xH2, xHp, chunk, final_ ? 1 : 0, out_chi_pe,
                                                        out_fh2, out_Nc);
  return cudaGetLastError();
}

cudaError_t launch_pdr_ntrans(const PdrSlabs& g, const double* xH2, double* Ntr, cudaStream_t st) {
  k_pdr_ntrans<<<(g.nslab + 63) / 64, 64, 0, st>>>(g, xH2, Ntr);
  return cudaGetLastError();
}

}  // namespace tcg
