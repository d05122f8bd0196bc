// Tensor-core inference of the seed network for the 32 cells of a warp (one per lane).
//
// Every layer is a 32 x 64 (cells x outputs) product computed with the warp-level BF16
// tensor-core instruction mma.sync.aligned.m16n8k16 (FP32 accumulate): two m16 tiles of
// cells, eight n8 tiles of outputs, k16 steps over the inputs.  The accumulator
// fragment of two neighbouring n8 tiles has exactly the register layout of the A
// fragment of one k16 step of the next layer (rows = cells, columns = features), so the
// activations never leave registers: bias, SiLU and the rounding to BF16 are applied to
// the accumulators, which then feed the next layer.  Only the first layer's inputs (each
// lane's own 13 features) and the last layer's 3 outputs move between lanes, by
// shuffles.  The weights are read as B fragments from a [out][in] BF16 copy of the
// network (MlpMma, built from the blob at load time); each lane reads 8 bytes per
// fragment, a warp the whole 256-byte tile.
//
// Every lane of the warp must call mlp_infer_warp together (the instruction is
// warp-collective); lanes without a cell pass any finite features and ignore the result.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_mlp.cuh"

namespace tcg {

// Weights in the layout the B fragments read: W[out][in] row-major, inputs of the first
// layer padded to 16 and outputs of the last to 8 with zeros.
struct MlpMma {
  float mean[MLP_INP], inv_std[MLP_INP];
  float b1[MLP_HID], b2[MLP_HID], b3[MLP_HID], b4[8];
  __nv_bfloat16 W1[MLP_HID * MLP_INP];
  __nv_bfloat16 W2[MLP_HID * MLP_HID];
  __nv_bfloat16 W3[MLP_HID * MLP_HID];
  __nv_bfloat16 W4[8 * MLP_HID];
};

// Builds the MlpMma copy of blob `w` on the device (tc_mlp.cu); stream-ordered.
cudaError_t mlp_mma_layout(const MlpDev* w, MlpMma* m, cudaStream_t st);

// D += A (16x16, row) * B (16x8, col), BF16 inputs, FP32 accumulators.
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Two floats rounded to BF16 and packed, the first in the low half (the element of the
// smaller column, as the fragments order them).
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float silu_fast(float z) { return z / (1.0f + __expf(-z)); }

// One hidden layer: A holds the input fragments [m-tile][k-step][4] (KS k-steps of 16
// inputs); W is [64][16 KS] BF16; the outputs after bias and SiLU become the next
// layer's input fragments Aout[m-tile][4 k-steps][4].
template <int KS>
__device__ __forceinline__ void mma_layer(const uint32_t (&A)[2][KS][4], const __nv_bfloat16* __restrict__ W,
                                          const float* __restrict__ b, uint32_t (&Aout)[2][4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int np = 0; np < 4; ++np) {  // a pair of n8 tiles = one k16 step of the next layer
    float acc[2][2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int col = 8 * (2 * np + q) + 2 * t;
      const float b0 = b[col], b1 = b[col + 1];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        acc[mt][q][0] = b0; acc[mt][q][1] = b1; acc[mt][q][2] = b0; acc[mt][q][3] = b1;
      }
    }
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const __nv_bfloat16* row = W + (size_t)(8 * (2 * np + q) + g) * (16 * KS) + 16 * ks + 2 * t;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_16816(acc[mt][q], A[mt][ks], b0, b1);
      }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      Aout[mt][np][0] = pack_bf16(silu_fast(acc[mt][0][0]), silu_fast(acc[mt][0][1]));
      Aout[mt][np][1] = pack_bf16(silu_fast(acc[mt][0][2]), silu_fast(acc[mt][0][3]));
      Aout[mt][np][2] = pack_bf16(silu_fast(acc[mt][1][0]), silu_fast(acc[mt][1][1]));
      Aout[mt][np][3] = pack_bf16(silu_fast(acc[mt][1][2]), silu_fast(acc[mt][1][3]));
    }
  }
}

// Network outputs o[3] for this lane's raw features f[MLP_IN]; all 32 lanes call it.
__device__ __forceinline__ void mlp_infer_warp(const MlpMma* __restrict__ m, const float* f, float* o) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // this lane's normalised features as 8 packed BF16 pairs (inputs 13..15 are zero)
  uint32_t w[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float x0 = (2 * j < MLP_IN) ? (f[2 * j] - m->mean[2 * j]) * m->inv_std[2 * j] : 0.f;
    const float x1 = (2 * j + 1 < MLP_IN) ? (f[2 * j + 1] - m->mean[2 * j + 1]) * m->inv_std[2 * j + 1] : 0.f;
    w[j] = pack_bf16(x0, x1);
  }
  // first layer's A fragments: row r of m-tile mt is the cell of lane 16 mt + r
  uint32_t A1[2][1][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = 16 * mt + g, r1 = r0 + 8;
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t v0 = __shfl_sync(FULL, w[j], r0);
      const uint32_t v1 = __shfl_sync(FULL, w[j], r1);
      if (j == t) { a0 = v0; a1 = v1; }
      if (j == t + 4) { a2 = v0; a3 = v1; }
    }
    A1[mt][0][0] = a0; A1[mt][0][1] = a1; A1[mt][0][2] = a2; A1[mt][0][3] = a3;
  }
  uint32_t H1[2][4][4], H2[2][4][4];
  mma_layer<1>(A1, m->W1, m->b1, H1);
  mma_layer<4>(H1, m->W2, m->b2, H2);
  mma_layer<4>(H2, m->W3, m->b3, H1);
  // output layer: one n8 tile (outputs 0..2 used)
  float acc[2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    acc[mt][0] = m->b4[2 * t]; acc[mt][1] = m->b4[2 * t + 1];
    acc[mt][2] = m->b4[2 * t]; acc[mt][3] = m->b4[2 * t + 1];
  }
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const __nv_bfloat16* row = m->W4 + (size_t)g * MLP_HID + 16 * ks + 2 * t;
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
    const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) mma_16816(acc[mt], H1[mt][ks], b0, b1);
  }
  // cell of lane L sits in m-tile L / 16, row L % 16 = g' (+8 in the upper half); its
  // outputs 0 and 1 are held by lane 4 g', output 2 by lane 4 g' + 1
  const int mt_me = lane >> 4, rr = lane & 15, gs = rr & 7, hi = rr >> 3;
  float r[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float v0 = __shfl_sync(FULL, acc[mt][2 * h], 4 * gs);
      const float v1 = __shfl_sync(FULL, acc[mt][2 * h + 1], 4 * gs);
      const float v2 = __shfl_sync(FULL, acc[mt][2 * h], 4 * gs + 1);
      if (mt == mt_me && h == hi) { r[0] = v0; r[1] = v1; r[2] = v2; }
    }
  o[0] = r[0];
  o[1] = r[1];
  o[2] = r[2];
}

}  // namespace tcg
