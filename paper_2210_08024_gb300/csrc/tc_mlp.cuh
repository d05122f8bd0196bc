// Seed network of the implicit solve: layout of its weights in the blob that
// tc_load_mlp accepts (the step kernel's tensor-core inference reads a re-laid-out copy,
// tc_mlp_mma.cuh).
//
// The network maps a cell's state, fields, metallicity, step length and the
// explicit-Euler changes over the step (13 features) through three hidden layers of 64
// SiLU units to 3 outputs: the changes over one backward-Euler step of length dt (the
// root the implicit solve looks for) minus the explicit-Euler ones,
//   o0 ~ (x_H2' - x_H2) / 0.5 - g0,  o1 ~ x_H+' - x_H+ - g1,  o2 ~ log10 T' - log10 T - g2,
// with g = dt (C_H2 / 0.5, C_H+, H / (K T_mu ln 10)) from the source terms at the start.
// Features: log10 n, log10 T, x_H2, x_H+, log10 chi_FUV, log10 f_shld,H2,
// log10(F_LyC + 1), log10 xi_cr, log10 dt, log10 Z'_d, g0, g1, g2; each normalised as
// (f - mean) * inv_std.
// Weights are BF16, everything else FP32; sums accumulate in FP32.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace tcg {

constexpr int MLP_IN = 13, MLP_HID = 64, MLP_OUT = 3;
constexpr int MLP_INP = 16;   // padded input width of W1
constexpr uint32_t MLP_MAGIC = 0x4C4D4354u;  // "TCML"
constexpr uint32_t MLP_VERSION = 3u;   // 3: thirteen inputs (explicit-Euler changes added)

// Weights are stored transposed ([in][out]).
struct MlpDev {
  uint32_t magic, version, n_in, n_hid, n_out, bytes, pad0, pad1;
  float in_mean[MLP_INP];
  float in_inv_std[MLP_INP];
  __nv_bfloat16 W1t[MLP_INP * MLP_HID];   // [k][j], rows k >= MLP_IN zero
  __nv_bfloat16 W2t[MLP_HID * MLP_HID];   // [k][j]
  __nv_bfloat16 W3t[MLP_HID * MLP_HID];   // [k][j]
  __nv_bfloat16 W4t[MLP_HID * 4];         // [k][m], column 3 zero
  float b1[MLP_HID], b2[MLP_HID], b3[MLP_HID], b4[4];
};
static_assert(sizeof(MlpDev) % 16 == 0, "MlpDev must stay 16-byte sized");

// SiLU activation of the hidden layers, z / (1 + e^-z).
__host__ __device__ __forceinline__ float mlp_silu(float z) {
#ifdef __CUDA_ARCH__
  return z / (1.0f + __expf(-z));
#else
  return z / (1.0f + expf(-z));
#endif
}

}  // namespace tcg
