// df64 (double-float) arithmetic on the device, built like the mixed step kernels (fast
// FP32 intrinsics, flush-to-zero): element-wise evaluation for the accuracy tests and
// throughput chains for the roofline of the mixed step (declared in include/tc_peak.h).
#include <cuda_runtime.h>

#include "../../include/tc.h"
#include "../../include/tc_peak.h"
#include "tc_df64.cuh"

namespace {
using tcg::df64;

__global__ void k_df64_eval(int op, const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const df64 x(a[i]);
    const df64 y(b ? b[i] : 0.0);
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

constexpr int CH = 8;

// kind 9: df64 multiply-add chains v = v a + b; kind 10: df64 exp chains v = exp(-v)
template <int KIND>
__global__ void k_df64_peak(int iters, double* sink) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  df64 v[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) v[c] = df64(0.5 + 1e-3 * (double)((tid + c) & 63));
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

// The df64 kinds of tc_peak_launch (tc_peak.cu forwards them here).
namespace tcg {
int df64_peak_launch(int kind, int grid, int block, int iters, double* sink, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == 9) k_df64_peak<9><<<grid, block, 0, st>>>(iters, sink);
  else if (kind == 10) k_df64_peak<10><<<grid, block, 0, st>>>(iters, sink);
  else return TC_EINVAL;
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ECUDA;
}
}  // namespace tcg
