// Seed network of the implicit solve: layout of its weights on the device and the
// per-lane inference used inside the step kernel.
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
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace tcg {

constexpr int MLP_IN = 13, MLP_HID = 64, MLP_OUT = 3;
constexpr int MLP_INP = 16;   // padded input width of W1
constexpr uint32_t MLP_MAGIC = 0x4C4D4354u;  // "TCML"
constexpr uint32_t MLP_VERSION = 3u;   // 3: thirteen inputs (explicit-Euler changes added)

// Weights are stored transposed ([in][out]) so that one input's weights for 16
// consecutive outputs are contiguous (two 16-byte loads, broadcast to the warp).
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

// Inference is host+device so that the host build of the step functions can run the
// seeded modes too.
#define TCG_MLP_FN __host__ __device__ __forceinline__

TCG_MLP_FN float mlp_silu(float z) {
#ifdef __CUDA_ARCH__
  return z / (1.0f + __expf(-z));
#else
  return z / (1.0f + expf(-z));
#endif
}

// Activation storage: FP32, or FP16 where shared memory is short (the step kernel).
TCG_MLP_FN float act_load(const float* p) { return *p; }
TCG_MLP_FN void act_store(float* p, float v) { *p = v; }
TCG_MLP_FN float act_load(const __half* p) { return __half2float(*p); }
TCG_MLP_FN void act_store(__half* p, float v) { *p = __float2half(v); }

// One hidden layer for this thread: out[j] = silu(b[j] + sum_k Wt[k][j] in[k]), with
// in[k] at in + k * st and out[j] at out + j * st.
template <int K, class A>
TCG_MLP_FN void mlp_layer(const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ b,
                                          const A* in, A* out, int st) {
#pragma unroll 1
  for (int j0 = 0; j0 < MLP_HID; j0 += 16) {
    float acc[16];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) acc[jj] = b[j0 + jj];
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const float a = act_load(in + k * st);
      const __nv_bfloat162* w2 = reinterpret_cast<const __nv_bfloat162*>(Wt + k * MLP_HID + j0);
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const float2 w = __bfloat1622float2(w2[jj]);
        acc[2 * jj] = fmaf(w.x, a, acc[2 * jj]);
        acc[2 * jj + 1] = fmaf(w.y, a, acc[2 * jj + 1]);
      }
    }
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) act_store(out + (j0 + jj) * st, mlp_silu(acc[jj]));
  }
}

// Network output for raw features f[MLP_IN].  `w` points to the weights; buf0/buf1 point
// to this thread's two activation buffers of 64 entries at stride `st`.
template <class A>
TCG_MLP_FN void mlp_infer(const MlpDev* w, A* buf0, A* buf1, int st, const float* f, float* o) {
#pragma unroll
  for (int k = 0; k < MLP_IN; ++k) act_store(buf1 + k * st, (f[k] - w->in_mean[k]) * w->in_inv_std[k]);
  mlp_layer<MLP_IN>(w->W1t, w->b1, buf1, buf0, st);
  mlp_layer<MLP_HID>(w->W2t, w->b2, buf0, buf1, st);
  mlp_layer<MLP_HID>(w->W3t, w->b3, buf1, buf0, st);
  float a0 = w->b4[0], a1 = w->b4[1], a2 = w->b4[2];
#pragma unroll 8
  for (int k = 0; k < MLP_HID; ++k) {
    const float h = act_load(buf0 + k * st);
    a0 = fmaf(__bfloat162float(w->W4t[k * 4 + 0]), h, a0);
    a1 = fmaf(__bfloat162float(w->W4t[k * 4 + 1]), h, a1);
    a2 = fmaf(__bfloat162float(w->W4t[k * 4 + 2]), h, a2);
  }
  o[0] = a0;
  o[1] = a1;
  o[2] = a2;
}

}  // namespace tcg
