// df64 (double-float) arithmetic on the device, built like the mixed step kernels (fast
// FP32 intrinsics, flush-to-zero): element-wise evaluation and the physics' source terms
// in df64 against FP64, for the accuracy tests, and throughput chains for the roofline
// of the mixed step (declared in include/tc_peak.h).
#include <cuda_runtime.h>

#include "../../include/tc.h"
#include "../../include/tc_peak.h"
#include "tc_launch.h"

namespace {
using tcg::df64;

__global__ void k_df64_eval(int op, const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const df64 x = tcg::to_df64(a[i]);
    const df64 y = tcg::to_df64(b ? b[i] : 0.0);
    df64 r;
    switch (op) {
      case 0: r = x + y; break;
      case 1: r = x * y; break;
      case 2: r = x / y; break;
      case 3: r = tcg::m_sqrt(x); break;
      case 4: r = tcg::m_exp(x); break;
      default: r = tcg::m_log(x); break;
    }
    out[i] = double(r);
  }
}

// Per cell at its stored state: the source terms in df64 against FP64 (errors as in
// include/tc_peak.h, tc_df64_source_check), SoA in err[5 n].
__global__ void __launch_bounds__(64) k_df64_source_check(tcg::DevFields f, tcg::DevParams p, double* err) {
  using namespace tcg;
  const long long n = f.ncell;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    CellC<double> c;
    double T, x2, xp;
    load_cell(f, i, p, c, T, x2, xp);
    const CellC<df64> cd = cast_cell<df64>(c);
    const double xH = 1.0 - 2.0 * x2 - xp;
    const ChemT<double> b = chem_T(c, T, p.flags);
    const CoolT<double> k = cool_T(c, b, p.flags);
    const Equil<double> q = equilibrium(c, b, x2, xp, -1.0);
    const Src<double> s = source(c, b, k, x2, xp, xH, q, -1.0, -1.0);
    const ChemT<df64> bd = chem_T(cd, to_df64(T), p.flags);
    const CoolT<df64> kd = cool_T(cd, bd, p.flags);
    const Equil<df64> qd = equilibrium(cd, bd, to_df64(x2), to_df64(xp), df64(-1.0));
    const Src<df64> sd = source(cd, bd, kd, to_df64(x2), to_df64(xp), to_df64(xH), qd, df64(-1.0), df64(-1.0));
    const double nn = c.n;
    err[i] = fabs(double(sd.H) - s.H) / (nn * fabs(s.G) + nn * nn * fabs(s.L));
    err[n + i] = fabs(double(sd.CH2) - s.CH2) / fmax(s.form + s.dest, 1e-300);
    err[2 * n + i] = fabs(double(sd.CHp) - s.CHp) / fmax(s.ion + s.rec, 1e-300);
    err[3 * n + i] = fabs(double(sd.Td) - s.Td) / s.Td;
    err[4 * n + i] = fabs(double(qd.xe) - q.xe) / q.xe;
  }
}

constexpr int CH = 8;

// kind 9: df64 multiply-add chains v = v a + b; kind 10: df64 exp chains v = exp(-v)
template <int KIND>
__global__ void k_df64_peak(int iters, double* sink) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  df64 v[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) v[c] = tcg::to_df64(0.5 + 1e-3 * (double)((tid + c) & 63));
  const df64 a(0.999), b(1e-4);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) v[c] = (KIND == 9) ? v[c] * a + b : tcg::m_exp(-v[c]);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += double(v[c]);
  sink[tid] = s;
}
}  // namespace

extern "C" int tc_df64_eval(int op, const double* a, const double* b, double* out, long long n, void* stream) {
  if (op < 0 || op > 5 || n < 0 || (n > 0 && (!a || !out)) || (op <= 2 && n > 0 && !b)) return TC_EINVAL;
  if (n == 0) return TC_OK;
  const int block = 256;
  const long long want = (n + block - 1) / block;
  const int grid = (int)(want < 4096 ? want : 4096);
  k_df64_eval<<<grid, block, 0, (cudaStream_t)stream>>>(op, a, b, out, n);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ECUDA;
}

namespace tcg {
cudaError_t launch_df64_source_check(const DevFields& f, const DevParams& p, double* err, cudaStream_t st) {
  const long long want = (f.ncell + 63) / 64;
  const int grid = (int)(want < 8192 ? want : 8192);
  k_df64_source_check<<<grid, 64, 0, st>>>(f, p, err);
  return cudaGetLastError();
}

// The df64 kinds of tc_peak_launch (tc_peak.cu forwards them here).
int df64_peak_launch(int kind, int grid, int block, int iters, double* sink, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == 9) k_df64_peak<9><<<grid, block, 0, st>>>(iters, sink);
  else if (kind == 10) k_df64_peak<10><<<grid, block, 0, st>>>(iters, sink);
  else return TC_EINVAL;
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ECUDA;
}
}  // namespace tcg
