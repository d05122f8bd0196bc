// Six-ray radiation fields, H2 self-shielding and CR attenuation (Secs. 5.2, 5.3;
// include/tc_sixray.h).
//
// Three passes, one per axis; each adds the two rays along its axis to per-cell
// accumulators held in the output arrays and the last one turns them into the fields:
//   acc.Nmin (in xi_cr)      smallest ray column seen so far
//   acc.Spe  (in chi_pe)     sum of exp(-sigma_PE (N_ray - Nmin))
//   acc.Slw  (in chi_lw)     sum of exp(-sigma_LW (N_ray - Nmin))
//   acc.Sh2  (in f_shld_h2)  sum of exp(-sigma_LW (N_ray - Nmin)) f_shld,H2(N_H2,ray)
// A ray's column is the sum of n dx over the cells between its entry face and the cell,
// accumulated from that face (exclusive scans in both directions; a line total minus a
// prefix would cancel to rounding noise near the far face, which the H2 self-shielding
// factor resolves in its Doppler-core regime).
//  * z and y passes: lines run across rows, so 32 neighbouring lines (consecutive x)
//    form a warp and loads stay coalesced; each line is cut into 8 segments scanned by
//    8 warps of a block, which combine their segment sums in shared memory (a two-level
//    scan), so even a 128^3 grid gives 131k threads.  Each segment is swept forwards
//    (the ray entering at the low face) and backwards (the ray entering at the high face).
//  * x pass: a line is a contiguous row; one warp scans it in chunks of 32 with shuffles,
//    backwards first, then forwards, where it also converts the accumulators.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/tc_sixray.h"

namespace tcg {
namespace {

constexpr double N0_CRATT = 9.35e20;  // Eq. e:cratt
constexpr int SEG = 8;                // segments per line in the z and y passes

struct SrConst {
  double dx, spe, slw, chi0, xi0;
};

// Eq. e:fshld_H2_DB with b_5 = 3 and x = N_H2 / 5e14 cm^-2.
__device__ __forceinline__ double f_shld_db(double N_h2) {
  const double x = N_h2 / 5e14;
  const double s = sqrt(1.0 + x);
  const double q = 1.0 + x / 3.0;
  return 0.965 / (q * q) + 0.035 / s * exp(-8.5e-4 * s);
}

// (1 - e^-t)/t, the cell average of e^-s over optical depth t.
__device__ __forceinline__ double cell_average(double t) {
  return (t < 1e-8) ? 1.0 - 0.5 * t : -expm1(-t) / t;
}

struct Acc {
  double Nmin, Spe, Slw, Sh2;
};

// Adds one ray with dust column N and H2 column NH2c to the cell centre.  The LW
// weight is the PE weight to the power sigma_LW / sigma_PE = 1.5.
__device__ __forceinline__ void add_ray(Acc& a, const SrConst& k, double N, double NH2c) {
  const double f = f_shld_db(NH2c);
  if (a.Spe == 0.0) {
    a.Nmin = N;
  } else if (N < a.Nmin) {
    const double r = exp(-k.spe * (a.Nmin - N));
    const double r15 = r * sqrt(r);
    a.Spe *= r;
    a.Slw *= r15;
    a.Sh2 *= r15;
    a.Nmin = N;
  }
  const double p = exp(-k.spe * (N - a.Nmin));
  const double q = p * sqrt(p);
  a.Spe += p;
  a.Slw += q;
  a.Sh2 += q * f;
}

__device__ __forceinline__ Acc load_acc(const double* chi_pe, const double* chi_lw, const double* fh2,
                                        const double* xi, long long c) {
  return Acc{xi[c], chi_pe[c], chi_lw[c], fh2[c]};
}

__device__ __forceinline__ void store_acc(double* chi_pe, double* chi_lw, double* fh2, double* xi, long long c,
                                          const Acc& a) {
  xi[c] = a.Nmin;
  chi_pe[c] = a.Spe;
  chi_lw[c] = a.Slw;
  fh2[c] = a.Sh2;
}

// Lines along z (FIRST = true: accumulators start empty) or y.  Block = 32 lanes
// (consecutive x) x SEG segment warps; blockIdx.x = x-tile + ntile * other, where
// other is y (z pass) or z (y pass).
template <bool FIRST>
__global__ void __launch_bounds__(32 * SEG) k_sr_lines(long long nx, long long len, long long lstride,
                                                      long long ostride, long long ntile, SrConst k,
                                                      const double* __restrict__ n, const double* __restrict__ xh2,
                                                      double* chi_pe, double* chi_lw, double* fh2, double* xi) {
  __shared__ double sN[SEG][32], sH[SEG][32];
  const int lane = threadIdx.x, seg = threadIdx.y;
  const long long tile = blockIdx.x % ntile, other = blockIdx.x / ntile;
  const long long i = tile * 32 + lane;
  const bool live = i < nx;
  const long long base = i + other * ostride;
  const long long c0 = len * seg / SEG, c1 = len * (seg + 1) / SEG;
  double sn = 0.0, sh = 0.0;
  if (live)
    for (long long c = c0; c < c1; ++c) {
      const long long e = base + c * lstride;
      sn += n[e] * k.dx;
      sh += (xh2[e] * n[e]) * k.dx;
    }
  sN[seg][lane] = sn;
  sH[seg][lane] = sh;
  __syncthreads();
  // columns of the segments before this one (from the low face) and after it (from the
  // high face)
  double fN = 0.0, fH = 0.0, bN = 0.0, bH = 0.0;
  for (int s = 0; s < seg; ++s) { fN += sN[s][lane]; fH += sH[s][lane]; }
  for (int s = SEG - 1; s > seg; --s) { bN += sN[s][lane]; bH += sH[s][lane]; }
  if (!live) return;
  for (long long c = c0; c < c1; ++c) {
    const long long e = base + c * lstride;
    const double nn = n[e];
    const double ownN = nn * k.dx;
    const double ownH = (xh2[e] * nn) * k.dx;
    const double half = 0.5 * xh2[e] * nn * k.dx;
    Acc a;
    if (FIRST) a = Acc{0.0, 0.0, 0.0, 0.0};
    else a = load_acc(chi_pe, chi_lw, fh2, xi, e);
    add_ray(a, k, fN, fH + half);
    store_acc(chi_pe, chi_lw, fh2, xi, e, a);
    fN += ownN;
    fH += ownH;
  }
  for (long long c = c1 - 1; c >= c0; --c) {
    const long long e = base + c * lstride;
    const double nn = n[e];
    const double ownN = nn * k.dx;
    const double ownH = (xh2[e] * nn) * k.dx;
    const double half = 0.5 * xh2[e] * nn * k.dx;
    Acc a = load_acc(chi_pe, chi_lw, fh2, xi, e);
    add_ray(a, k, bN, bH + half);
    store_acc(chi_pe, chi_lw, fh2, xi, e, a);
    bN += ownN;
    bH += ownH;
  }
}

// Rows along x: one warp per row, chunks of 32 cells scanned with shuffles: the ray
// entering at the high face first (suffix scans, last chunk first), then the ray
// entering at the low face (prefix scans), which also converts the accumulators into
// the fields.
__global__ void __launch_bounds__(256) k_sr_rows(long long nx, long long nrows, SrConst k,
                                                 const double* __restrict__ n, const double* __restrict__ xh2,
                                                 double* chi_pe, double* chi_lw, double* fh2, double* xi,
                                                 double* Neff) {
  const long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nrows) return;
  const long long base = row * nx;
  const long long nchunk = (nx + 31) / 32;
  double carryN = 0.0, carryH = 0.0;
  for (long long ch = nchunk - 1; ch >= 0; --ch) {
    const long long i = ch * 32 + lane;
    const bool live = i < nx;
    const double nn = live ? n[base + i] : 0.0;
    const double xx = live ? xh2[base + i] : 0.0;
    double iN = nn * k.dx, iH = (xx * nn) * k.dx;  // inclusive suffix scan within the chunk
    for (int d = 1; d < 32; d <<= 1) {
      const double vN = __shfl_down_sync(0xffffffffu, iN, d);
      const double vH = __shfl_down_sync(0xffffffffu, iH, d);
      if (lane + d < 32) { iN += vN; iH += vH; }
    }
    double eN = __shfl_down_sync(0xffffffffu, iN, 1), eH = __shfl_down_sync(0xffffffffu, iH, 1);
    if (lane == 31) { eN = 0.0; eH = 0.0; }
    const double chunkN = __shfl_sync(0xffffffffu, iN, 0), chunkH = __shfl_sync(0xffffffffu, iH, 0);
    if (live) {
      const long long e = base + i;
      const double half = 0.5 * xx * nn * k.dx;
      Acc a = load_acc(chi_pe, chi_lw, fh2, xi, e);
      add_ray(a, k, carryN + eN, carryH + eH + half);
      store_acc(chi_pe, chi_lw, fh2, xi, e, a);
    }
    carryN += chunkN;
    carryH += chunkH;
  }
  carryN = 0.0;
  carryH = 0.0;
  for (long long i0 = 0; i0 < nx; i0 += 32) {
    const long long i = i0 + lane;
    const bool live = i < nx;
    const double nn = live ? n[base + i] : 0.0;
    const double xx = live ? xh2[base + i] : 0.0;
    double iN = nn * k.dx, iH = (xx * nn) * k.dx;  // inclusive prefix scan within the chunk
    for (int d = 1; d < 32; d <<= 1) {
      const double vN = __shfl_up_sync(0xffffffffu, iN, d);
      const double vH = __shfl_up_sync(0xffffffffu, iH, d);
      if (lane >= d) { iN += vN; iH += vH; }
    }
    double eN = __shfl_up_sync(0xffffffffu, iN, 1), eH = __shfl_up_sync(0xffffffffu, iH, 1);
    if (lane == 0) { eN = 0.0; eH = 0.0; }
    const double chunkN = __shfl_sync(0xffffffffu, iN, 31), chunkH = __shfl_sync(0xffffffffu, iH, 31);
    if (live) {
      const long long e = base + i;
      const double half = 0.5 * xx * nn * k.dx;
      Acc a = load_acc(chi_pe, chi_lw, fh2, xi, e);
      add_ray(a, k, carryN + eN, carryH + eH + half);
      // fields of the cell
      const double gpe = cell_average(k.spe * nn * k.dx);
      const double glw = cell_average(k.slw * nn * k.dx);
      chi_pe[e] = k.chi0 / 6.0 * exp(-k.spe * a.Nmin) * a.Spe * gpe;
      chi_lw[e] = k.chi0 / 6.0 * exp(-k.slw * a.Nmin) * a.Slw * glw;
      fh2[e] = a.Sh2 / a.Slw;
      double ne = 0.0;
      if (k.spe > 0.0) ne = (k.spe * a.Nmin - log(a.Spe * gpe / 6.0)) / k.spe;
      xi[e] = (ne <= N0_CRATT) ? k.xi0 : k.xi0 * N0_CRATT / ne;
      if (Neff) Neff[e] = ne;
    }
    carryN += chunkN;
    carryH += chunkH;
  }
}

bool al8(const void* p) { return (((unsigned long long)p) & 7ull) == 0; }

}  // namespace
}  // namespace tcg

extern "C" int tc_sixray(const tc_sixray_grid* g, const double* n, const double* x_h2, double* chi_pe,
                         double* chi_lw, double* f_shld_h2, double* xi_cr, double* N_eff, void* stream) {
  using namespace tcg;
  if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return TC_EINVAL;
  if (!(g->dx_cm > 0.0) || !isfinite(g->dx_cm) || !(g->chi0 >= 0.0) || !(g->xi0 >= 0.0) || !(g->Zd >= 0.0) ||
      !isfinite(g->chi0) || !isfinite(g->xi0) || !isfinite(g->Zd))
    return TC_EINVAL;
  const double ncell_d = (double)g->nx * (double)g->ny * (double)g->nz;
  if (ncell_d > 4.0e12) return TC_EINVAL;
  const void* ptrs[] = {n, x_h2, chi_pe, chi_lw, f_shld_h2, xi_cr};
  for (const void* p : ptrs)
    if (!p || !al8(p)) return TC_EINVAL;
  if (N_eff && !al8(N_eff)) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  SrConst k;
  k.dx = g->dx_cm;
  k.spe = 1.0e-21 * g->Zd;
  k.slw = 1.5e-21 * g->Zd;
  k.chi0 = g->chi0;
  k.xi0 = g->xi0;
  const long long nx = g->nx, ny = g->ny, nz = g->nz;
  const long long ntile = (nx + 31) / 32;
  const dim3 blk(32, SEG);
  // z lines: other = y (stride nx), line stride nx*ny
  long long nb = ntile * ny;
  if (nb > 2147483647LL) return TC_EINVAL;
  k_sr_lines<true><<<(unsigned)nb, blk, 0, st>>>(nx, nz, nx * ny, nx, ntile, k, n, x_h2, chi_pe, chi_lw, f_shld_h2,
                                                 xi_cr);
  if (cudaGetLastError() != cudaSuccess) return TC_ECUDA;
  // y lines: other = z (stride nx*ny), line stride nx
  nb = ntile * nz;
  if (nb > 2147483647LL) return TC_EINVAL;
  k_sr_lines<false><<<(unsigned)nb, blk, 0, st>>>(nx, ny, nx, nx * ny, ntile, k, n, x_h2, chi_pe, chi_lw, f_shld_h2,
                                                  xi_cr);
  if (cudaGetLastError() != cudaSuccess) return TC_ECUDA;
  // x rows
  const long long nrows = ny * nz;
  nb = (nrows + 7) / 8;
  if (nb > 2147483647LL) return TC_EINVAL;
  k_sr_rows<<<(unsigned)nb, 256, 0, st>>>(nx, nrows, k, n, x_h2, chi_pe, chi_lw, f_shld_h2, xi_cr, N_eff);
  if (cudaGetLastError() != cudaSuccess) return TC_ECUDA;
  return TC_OK;
}
