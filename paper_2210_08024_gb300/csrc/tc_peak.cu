// Pipe-throughput microbenchmarks (declared in include/tc_peak.h): independent
// dependency chains per thread so that the pipe, not latency, bounds the rate.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/tc.h"
#include "../../include/tc_peak.h"

namespace tcg {
int df64_peak_launch(int kind, int grid, int block, int iters, double* sink, void* stream);  // tc_df64_diag.cu
}

namespace {
constexpr int CH = 8;

template <int KIND>
__global__ void k_peak(int iters, double* sink) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (KIND == 1 || KIND == 7 || KIND == 8) {
    float v[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) v[c] = 0.5f + 1e-3f * (float)((tid + c) & 63);
    const float a = 0.999f, b = 1e-4f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CH; ++c) v[c] = (KIND == 1) ? fmaf(v[c], a, b) : (KIND == 7) ? expf(-v[c]) : __expf(-v[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += v[c];
    sink[tid] = (double)s;
  } else {
    double v[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) v[c] = 0.5 + 1e-3 * (double)((tid + c) & 63);
    const double a = 0.999, b = 1e-4;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        if (KIND == 0) v[c] = fma(v[c], a, b);
        if (KIND == 2) v[c] = exp(-v[c]);          // converges to the omega constant
        if (KIND == 3) v[c] = log(v[c] + 2.0);      // converges to ~1.146
        if (KIND == 4) v[c] = sqrt(v[c] + 1.0);     // converges to the golden ratio
        if (KIND == 5) v[c] = 1.0 / (v[c] + 1.0);   // converges to 0.618
        if (KIND == 6) v[c] = pow(v[c] + 1.0, 0.7);
      }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += v[c];
    sink[tid] = s;
  }
}
}  // namespace

extern "C" int tc_peak_chains(void) { return CH; }

extern "C" int tc_peak_launch(int kind, int grid, int block, int iters, double* sink, void* stream) {
  if (grid < 1 || block < 1 || block > 1024 || iters < 1 || !sink) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  switch (kind) {
    case 0: k_peak<0><<<grid, block, 0, st>>>(iters, sink); break;
    case 1: k_peak<1><<<grid, block, 0, st>>>(iters, sink); break;
    case 2: k_peak<2><<<grid, block, 0, st>>>(iters, sink); break;
    case 3: k_peak<3><<<grid, block, 0, st>>>(iters, sink); break;
    case 4: k_peak<4><<<grid, block, 0, st>>>(iters, sink); break;
    case 5: k_peak<5><<<grid, block, 0, st>>>(iters, sink); break;
    case 6: k_peak<6><<<grid, block, 0, st>>>(iters, sink); break;
    case 7: k_peak<7><<<grid, block, 0, st>>>(iters, sink); break;
    case 8: k_peak<8><<<grid, block, 0, st>>>(iters, sink); break;
    case 9:
    case 10: return tcg::df64_peak_launch(kind, grid, block, iters, sink, stream);
    default: return TC_EINVAL;
  }
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ECUDA;
}
