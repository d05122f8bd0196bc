// Training of the seed network on the GPU (declared in include/tc_mlp.h).
//
// Parameters live on the device as one FP32 master vector in the order
//   W1[64][13], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[3][64], b4[3]
// (weights [out][in]).  The forward and backward passes use the weights rounded to
// BF16, as the step kernel's inference does, and accumulate in FP32.  The weight
// gradient of the BF16 network is applied to the FP32 masters by Adam.
//
// One training step is a handful of small kernels, layer by layer: normalise ->
// dense+SiLU x3 -> dense -> loss -> back through each layer (input gradient, then
// weight gradient) -> Adam.  The network is tiny (9155 parameters), so these kernels
// are plain FP32 FMA loops; the time of the seeded solver is spent in the step kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/tc.h"
#include "../../include/tc_mlp.h"
#include "tc_mlp.cuh"
#include "tc_mlp_mma.cuh"

namespace tcg {
namespace {
// One block of 256 threads: the [out][in] copy of the blob's transposed weights that
// the tensor-core inference reads as B fragments (tc_mlp_mma.cuh).
__global__ void k_mlp_mma_layout(const MlpDev* __restrict__ w, MlpMma* __restrict__ m) {
  for (int i = threadIdx.x; i < MLP_INP; i += blockDim.x) {
    m->mean[i] = w->in_mean[i];
    m->inv_std[i] = w->in_inv_std[i];
  }
  for (int i = threadIdx.x; i < MLP_HID; i += blockDim.x) {
    m->b1[i] = w->b1[i];
    m->b2[i] = w->b2[i];
    m->b3[i] = w->b3[i];
  }
  for (int i = threadIdx.x; i < 8; i += blockDim.x) m->b4[i] = (i < MLP_OUT) ? w->b4[i] : 0.f;
  for (int i = threadIdx.x; i < MLP_HID * MLP_INP; i += blockDim.x) {
    const int o = i / MLP_INP, k = i % MLP_INP;
    m->W1[i] = w->W1t[k * MLP_HID + o];
  }
  for (int i = threadIdx.x; i < MLP_HID * MLP_HID; i += blockDim.x) {
    const int o = i / MLP_HID, k = i % MLP_HID;
    m->W2[i] = w->W2t[k * MLP_HID + o];
    m->W3[i] = w->W3t[k * MLP_HID + o];
  }
  for (int i = threadIdx.x; i < 8 * MLP_HID; i += blockDim.x) {
    const int o = i / MLP_HID, k = i % MLP_HID;
    m->W4[i] = (o < MLP_OUT) ? w->W4t[k * 4 + o] : __float2bfloat16_rn(0.f);
  }
}
}  // namespace

cudaError_t mlp_mma_layout(const MlpDev* w, MlpMma* m, cudaStream_t st) {
  k_mlp_mma_layout<<<1, 256, 0, st>>>(w, m);
  return cudaGetLastError();
}
}  // namespace tcg

namespace {

using tcg::MLP_HID;
using tcg::MLP_IN;
using tcg::MLP_OUT;

constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + 64 * MLP_IN, OFF_W2 = OFF_B1 + 64, OFF_B2 = OFF_W2 + 64 * 64,
              OFF_W3 = OFF_B2 + 64, OFF_B3 = OFF_W3 + 64 * 64, OFF_W4 = OFF_B3 + 64, OFF_B4 = OFF_W4 + 3 * 64,
              NPARAM = OFF_B4 + 3;

__device__ __forceinline__ float bf(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }
__device__ __forceinline__ float silu_d(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

__global__ void k_norm(const float* __restrict__ X, int B, const float* __restrict__ mean,
                       const float* __restrict__ inv_std, float* __restrict__ A0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * MLP_IN) return;
  const int k = i % MLP_IN;
  A0[i] = (X[i] - mean[k]) * inv_std[k];
}

// Z[b][n] = b[n] + sum_k bf16(W[n][k]) A[b][k]; H = silu(Z) when act.
__global__ void k_fwd(const float* __restrict__ A, int K, const float* __restrict__ W, const float* __restrict__ bias,
                      int N, int B, float* __restrict__ Z, float* __restrict__ H, bool act) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * N) return;
  const int b = i / N, n = i % N;
  float acc = bias[n];
  for (int k = 0; k < K; ++k) acc = fmaf(bf(W[n * K + k]), A[b * K + k], acc);
  Z[i] = acc;
  if (act) H[i] = tcg::mlp_silu(acc);
}

// G[b][m] = 2 w_m (O - Y) / B; loss += sum w_m (O - Y)^2 / B.
__global__ void k_loss(const float* __restrict__ O, const float* __restrict__ Y, int B, float w0, float w1, float w2,
                       float* __restrict__ G, float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < B * MLP_OUT) {
    const int m = i % MLP_OUT;
    const float w = (m == 0) ? w0 : (m == 1) ? w1 : w2;
    const float d = O[i] - Y[i];
    G[i] = 2.f * w * d / (float)B;
    l = w * d * d / (float)B;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

// Gin[b][k] = (sum_n Gout[b][n] bf16(W[n][k])) * silu'(Zin[b][k])
__global__ void k_bwd_data(const float* __restrict__ Gout, int N, const float* __restrict__ W, int K,
                           const float* __restrict__ Zin, int B, float* __restrict__ Gin) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * K) return;
  const int b = i / K, k = i % K;
  float acc = 0.f;
  for (int n = 0; n < N; ++n) acc = fmaf(Gout[b * N + n], bf(W[n * K + k]), acc);
  Gin[i] = acc * silu_d(Zin[i]);
}

// dW[n][k] = sum_b Gout[b][n] A[b][k]; db[n] = sum_b Gout[b][n].  One thread per (n, k)
// (plus one per n for the bias), each summing over a slice of the batch; slices are
// combined with atomicAdd.
__global__ void k_bwd_w(const float* __restrict__ Gout, int N, const float* __restrict__ A, int K, int B, int bslice,
                        float* __restrict__ dW, float* __restrict__ db) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int b0 = blockIdx.y * bslice;
  const int b1 = min(B, b0 + bslice);
  if (i < N * K) {
    const int n = i / K, k = i % K;
    float acc = 0.f;
    for (int b = b0; b < b1; ++b) acc = fmaf(Gout[b * N + n], A[b * K + k], acc);
    atomicAdd(&dW[i], acc);
  } else if (i < N * K + N) {
    const int n = i - N * K;
    float acc = 0.f;
    for (int b = b0; b < b1; ++b) acc += Gout[b * N + n];
    atomicAdd(&db[n], acc);
  }
}

__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline int blocks(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

struct tc_mlp {
  float* theta = nullptr;  // NPARAM masters
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* norm = nullptr;   // mean[MLP_IN], inv_std[MLP_IN]
  float* loss = nullptr;
  float* work = nullptr;   // activations for cap samples
  int cap = 0;
  long long t = 0;         // Adam step count
  float h_mean[MLP_IN], h_inv_std[MLP_IN];
};

namespace {

// Work layout for B samples: A0[B*MLP_IN] Z1 H1 Z2 H2 Z3 H3 [B*64 each] O G[B*3] G3 G2 G1 [B*64].
size_t work_floats(int B) { return (size_t)B * (MLP_IN + 6 * MLP_HID + 2 * MLP_OUT + 3 * MLP_HID); }

int ensure_cap(tc_mlp* h, int B) {
  if (B <= h->cap) return TC_OK;
  cudaFree(h->work);
  h->work = nullptr;
  h->cap = 0;
  if (cudaMalloc(&h->work, work_floats(B) * sizeof(float)) != cudaSuccess) return TC_ENOMEM;
  h->cap = B;
  return TC_OK;
}

struct Bufs {
  float *A0, *Z1, *H1, *Z2, *H2, *Z3, *H3, *O, *G, *G3, *G2, *G1;
};

Bufs bufs(tc_mlp* h, int B) {
  Bufs b;
  float* p = h->work;
  b.A0 = p; p += (size_t)B * MLP_IN;
  b.Z1 = p; p += (size_t)B * MLP_HID;
  b.H1 = p; p += (size_t)B * MLP_HID;
  b.Z2 = p; p += (size_t)B * MLP_HID;
  b.H2 = p; p += (size_t)B * MLP_HID;
  b.Z3 = p; p += (size_t)B * MLP_HID;
  b.H3 = p; p += (size_t)B * MLP_HID;
  b.O = p; p += (size_t)B * MLP_OUT;
  b.G = p; p += (size_t)B * MLP_OUT;
  b.G3 = p; p += (size_t)B * MLP_HID;
  b.G2 = p; p += (size_t)B * MLP_HID;
  b.G1 = p;
  return b;
}

int forward(tc_mlp* h, const float* X, int B, cudaStream_t st, Bufs& b) {
  const int T = 256;
  k_norm<<<blocks((long long)B * MLP_IN, T), T, 0, st>>>(X, B, h->norm, h->norm + MLP_IN, b.A0);
  k_fwd<<<blocks((long long)B * MLP_HID, T), T, 0, st>>>(b.A0, MLP_IN, h->theta + OFF_W1, h->theta + OFF_B1, MLP_HID,
                                                          B, b.Z1, b.H1, true);
  k_fwd<<<blocks((long long)B * MLP_HID, T), T, 0, st>>>(b.H1, MLP_HID, h->theta + OFF_W2, h->theta + OFF_B2, MLP_HID,
                                                          B, b.Z2, b.H2, true);
  k_fwd<<<blocks((long long)B * MLP_HID, T), T, 0, st>>>(b.H2, MLP_HID, h->theta + OFF_W3, h->theta + OFF_B3, MLP_HID,
                                                          B, b.Z3, b.H3, true);
  k_fwd<<<blocks((long long)B * MLP_OUT, T), T, 0, st>>>(b.H3, MLP_HID, h->theta + OFF_W4, h->theta + OFF_B4, MLP_OUT,
                                                          B, b.O, nullptr, false);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ECUDA;
}

int backward(tc_mlp* h, const float* Y, int B, const float* w3, cudaStream_t st, Bufs& b) {
  const int T = 256;
  if (cudaMemsetAsync(h->grad, 0, NPARAM * sizeof(float), st) != cudaSuccess) return TC_ECUDA;
  if (cudaMemsetAsync(h->loss, 0, sizeof(float), st) != cudaSuccess) return TC_ECUDA;
  const float w0 = w3 ? w3[0] : 1.f, w1 = w3 ? w3[1] : 1.f, w2 = w3 ? w3[2] : 1.f;
  k_loss<<<blocks((long long)B * MLP_OUT, T), T, 0, st>>>(b.O, Y, B, w0, w1, w2, b.G, h->loss);
  const int bs = 512;
  const int ns = (B + bs - 1) / bs;
  // output layer
  k_bwd_w<<<dim3(blocks(MLP_OUT * MLP_HID + MLP_OUT, T), ns), T, 0, st>>>(b.G, MLP_OUT, b.H3, MLP_HID, B, bs,
                                                                            h->grad + OFF_W4, h->grad + OFF_B4);
  k_bwd_data<<<blocks((long long)B * MLP_HID, T), T, 0, st>>>(b.G, MLP_OUT, h->theta + OFF_W4, MLP_HID, b.Z3, B, b.G3);
  // hidden layer 3
  k_bwd_w<<<dim3(blocks(MLP_HID * MLP_HID + MLP_HID, T), ns), T, 0, st>>>(b.G3, MLP_HID, b.H2, MLP_HID, B, bs,
                                                                            h->grad + OFF_W3, h->grad + OFF_B3);
  k_bwd_data<<<blocks((long long)B * MLP_HID, T), T, 0, st>>>(b.G3, MLP_HID, h->theta + OFF_W3, MLP_HID, b.Z2, B, b.G2);
  // hidden layer 2
  k_bwd_w<<<dim3(blocks(MLP_HID * MLP_HID + MLP_HID, T), ns), T, 0, st>>>(b.G2, MLP_HID, b.H1, MLP_HID, B, bs,
                                                                            h->grad + OFF_W2, h->grad + OFF_B2);
  k_bwd_data<<<blocks((long long)B * MLP_HID, T), T, 0, st>>>(b.G2, MLP_HID, h->theta + OFF_W2, MLP_HID, b.Z1, B, b.G1);
  // hidden layer 1
  k_bwd_w<<<dim3(blocks(MLP_HID * MLP_IN + MLP_HID, T), ns), T, 0, st>>>(b.G1, MLP_HID, b.A0, MLP_IN, B, bs,
                                                                           h->grad + OFF_W1, h->grad + OFF_B1);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ECUDA;
}

// splitmix64 (Steele, Lea & Flood 2014) for a reproducible weight initialisation.
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int tc_mlp_n_params(void) { return NPARAM; }

int tc_mlp_create(unsigned long long seed, tc_mlp** out) {
  if (!out) return TC_EINVAL;
  tc_mlp* h = new (std::nothrow) tc_mlp();
  if (!h) return TC_ENOMEM;
  bool ok = cudaMalloc(&h->theta, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->grad, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->m, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->v, NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->norm, 2 * MLP_IN * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->loss, sizeof(float)) == cudaSuccess;
  if (!ok) {
    tc_mlp_destroy(h);
    return TC_ENOMEM;
  }
  // Uniform initialisation with bound sqrt(6 / fan_in) (He et al. 2015), zero biases.
  std::vector<float> th(NPARAM, 0.f);
  uint64_t s = seed;
  auto fill = [&](int off, int nout, int nin) {
    const double bound = sqrt(6.0 / nin);
    for (int i = 0; i < nout * nin; ++i) {
      const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
      th[off + i] = (float)((2.0 * u - 1.0) * bound);
    }
  };
  fill(OFF_W1, 64, MLP_IN);
  fill(OFF_W2, 64, 64);
  fill(OFF_W3, 64, 64);
  fill(OFF_W4, 3, 64);
  for (int i = OFF_W4; i < OFF_W4 + 3 * 64; ++i) th[i] *= 0.1f;  // small initial outputs
  for (int k = 0; k < MLP_IN; ++k) { h->h_mean[k] = 0.f; h->h_inv_std[k] = 1.f; }
  float nrm[2 * MLP_IN];
  for (int k = 0; k < MLP_IN; ++k) { nrm[k] = 0.f; nrm[MLP_IN + k] = 1.f; }
  ok = cudaMemcpy(h->theta, th.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(h->m, 0, NPARAM * sizeof(float)) == cudaSuccess &&
       cudaMemset(h->v, 0, NPARAM * sizeof(float)) == cudaSuccess &&
       cudaMemcpy(h->norm, nrm, sizeof(nrm), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    tc_mlp_destroy(h);
    return TC_ECUDA;
  }
  *out = h;
  return TC_OK;
}

void tc_mlp_destroy(tc_mlp* h) {
  if (!h) return;
  cudaFree(h->theta);
  cudaFree(h->grad);
  cudaFree(h->m);
  cudaFree(h->v);
  cudaFree(h->norm);
  cudaFree(h->loss);
  cudaFree(h->work);
  delete h;
}

int tc_mlp_set_norm(tc_mlp* h, const float* mean, const float* stdev) {
  if (!h || !mean || !stdev) return TC_EINVAL;
  float nrm[2 * MLP_IN];
  for (int k = 0; k < MLP_IN; ++k) {
    if (!(stdev[k] > 0.f) || !isfinite(mean[k])) return TC_EINVAL;
    h->h_mean[k] = mean[k];
    h->h_inv_std[k] = 1.f / stdev[k];
    nrm[k] = h->h_mean[k];
    nrm[MLP_IN + k] = h->h_inv_std[k];
  }
  return cudaMemcpy(h->norm, nrm, sizeof(nrm), cudaMemcpyHostToDevice) == cudaSuccess ? TC_OK : TC_ECUDA;
}

int tc_mlp_set_params(tc_mlp* h, const float* theta) {
  if (!h || !theta) return TC_EINVAL;
  return cudaMemcpy(h->theta, theta, NPARAM * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess ? TC_OK
                                                                                                      : TC_ECUDA;
}

int tc_mlp_get_params(const tc_mlp* h, float* theta) {
  if (!h || !theta) return TC_EINVAL;
  return cudaMemcpy(theta, h->theta, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? TC_OK
                                                                                                      : TC_ECUDA;
}

int tc_mlp_predict(tc_mlp* h, const float* X, int B, float* out, void* stream) {
  if (!h || B < 0 || (B > 0 && (!X || !out))) return TC_EINVAL;
  if (B == 0) return TC_OK;
  int rc = ensure_cap(h, B);
  if (rc != TC_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Bufs b = bufs(h, B);
  rc = forward(h, X, B, st, b);
  if (rc != TC_OK) return rc;
  return cudaMemcpyAsync(out, b.O, (size_t)B * MLP_OUT * sizeof(float), cudaMemcpyDeviceToDevice, st) == cudaSuccess
             ? TC_OK : TC_ECUDA;
}

int tc_mlp_grad(tc_mlp* h, const float* X, const float* Y, int B, const float* w3, float* grad, float* loss,
                void* stream) {
  if (!h || B < 1 || !X || !Y) return TC_EINVAL;
  int rc = ensure_cap(h, B);
  if (rc != TC_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Bufs b = bufs(h, B);
  rc = forward(h, X, B, st, b);
  if (rc == TC_OK) rc = backward(h, Y, B, w3, st, b);
  if (rc != TC_OK) return rc;
  if (grad && cudaMemcpyAsync(grad, h->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return TC_ECUDA;
  if (loss && cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return TC_ECUDA;
  return TC_OK;
}

int tc_mlp_train_step(tc_mlp* h, const float* X, const float* Y, int B, const float* w3, float lr, float* loss,
                      void* stream) {
  int rc = tc_mlp_grad(h, X, Y, B, w3, nullptr, loss, stream);
  if (rc != TC_OK) return rc;
  h->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - (float)pow(b1, (double)h->t), c2 = 1.f - (float)pow(b2, (double)h->t);
  k_adam<<<blocks(NPARAM, 256), 256, 0, (cudaStream_t)stream>>>(h->theta, h->grad, h->m, h->v, NPARAM, lr, b1, b2,
                                                                 1e-8f, c1, c2);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ECUDA;
}

size_t tc_mlp_blob_bytes(void) { return sizeof(tcg::MlpDev); }

int tc_mlp_export(const tc_mlp* h, void* blob, size_t cap) {
  if (!h || !blob || cap < sizeof(tcg::MlpDev)) return TC_EINVAL;
  std::vector<float> th(NPARAM);
  if (cudaMemcpy(th.data(), h->theta, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return TC_ECUDA;
  tcg::MlpDev d;
  memset(&d, 0, sizeof(d));
  d.magic = tcg::MLP_MAGIC;
  d.version = tcg::MLP_VERSION;
  d.n_in = MLP_IN;
  d.n_hid = MLP_HID;
  d.n_out = MLP_OUT;
  d.bytes = (uint32_t)sizeof(tcg::MlpDev);
  for (int k = 0; k < tcg::MLP_INP; ++k) {
    d.in_mean[k] = (k < MLP_IN) ? h->h_mean[k] : 0.f;
    d.in_inv_std[k] = (k < MLP_IN) ? h->h_inv_std[k] : 0.f;
  }
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int i = 0; i < tcg::MLP_INP * MLP_HID; ++i) d.W1t[i] = zero;
  for (int i = 0; i < MLP_HID * 4; ++i) d.W4t[i] = zero;
  for (int j = 0; j < MLP_HID; ++j) {
    for (int k = 0; k < MLP_IN; ++k) d.W1t[k * MLP_HID + j] = __float2bfloat16_rn(th[OFF_W1 + j * MLP_IN + k]);
    for (int k = 0; k < MLP_HID; ++k) {
      d.W2t[k * MLP_HID + j] = __float2bfloat16_rn(th[OFF_W2 + j * MLP_HID + k]);
      d.W3t[k * MLP_HID + j] = __float2bfloat16_rn(th[OFF_W3 + j * MLP_HID + k]);
    }
    d.b1[j] = th[OFF_B1 + j];
    d.b2[j] = th[OFF_B2 + j];
    d.b3[j] = th[OFF_B3 + j];
  }
  for (int m = 0; m < MLP_OUT; ++m) {
    for (int k = 0; k < MLP_HID; ++k) d.W4t[k * 4 + m] = __float2bfloat16_rn(th[OFF_W4 + m * MLP_HID + k]);
    d.b4[m] = th[OFF_B4 + m];
  }
  d.b4[3] = 0.f;
  memcpy(blob, &d, sizeof(d));
  return TC_OK;
}

}  // extern "C"
