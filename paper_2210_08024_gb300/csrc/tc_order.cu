// Cost-ordered work queue (tc_params.order_cells).
//
// A cell's cost is dominated by its number of substeps, and the substep rule of Sec.
// 6.1 predicts it from the start state: a cell whose first substep is dts_1 needs
// about dt / dts_1 of them (rank correlation 0.999 with the actual count on the slab,
// 0.83 with the Newton iterations).  Handing cells to the persistent kernel longest
// first does two things: the few cells with hundreds of Newton iterations no longer
// start last and run alone at the end of the launch, and neighbouring lanes of a warp
// hold cells of similar cost.  On the 128^3 slab, perfect ordering took FP64 Newton from
// 511 to 331 ms and mixed from 352 to 177 ms.  Results do not depend on the order.
//
//   k_order_key      one thread per cell: initial C/O/e equilibrium, start-state sources
//                    (in FP32: they only pick a class), cost class, block histogram
//   k_order_scan     exclusive scan of the ORDER_BUCKETS counts (one warp)
//   k_order_scatter  one thread per cell: position = class offset + rank (warp-aggregated
//                    atomics); cells of one class keep no particular order
#include "tc_order.cuh"

namespace tcg {
namespace {

template <bool BATCH>
__device__ __forceinline__ void locate(const DevFields& f1, const BoxTable* boxes, long long gi, DevFields& fb,
                                       long long& li) {
  if (BATCH) {
    int lo = 0, hi = boxes->nbox - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (boxes->start[mid] <= gi) lo = mid; else hi = mid - 1;
    }
    fb = boxes->box[lo];
    li = gi - boxes->start[lo];
  } else {
    fb = f1;
    li = gi;
  }
}

template <bool BATCH>
__global__ void __launch_bounds__(128) k_order_key(DevFields f1, const BoxTable* __restrict__ boxes, DevParams p,
                                                   double dt, long long ntotal, unsigned char* __restrict__ key,
                                                   unsigned* __restrict__ hist) {
  __shared__ unsigned sh[ORDER_BUCKETS];
  for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < ntotal;
       gi += (long long)gridDim.x * blockDim.x) {
    DevFields fb;
    long long li;
    locate<BATCH>(f1, boxes, gi, fb, li);
    if (fb.hint) {
      // a caller's cost estimate (e.g. the previous step's Newton iterations): eighth
      // octaves of 1 + hint
      const double u = 8.0 * log2(1.0 + fmax((double)fb.hint[li], 0.0));
      const int bh = (u >= ORDER_BUCKETS - 1) ? ORDER_BUCKETS - 1 : (int)u;
      const int kh = ORDER_BUCKETS - 1 - bh;
      key[gi] = (unsigned char)kh;
      atomicAdd(&sh[kh], 1u);
      continue;
    }
    // The prediction only picks a quarter-octave class, so it is evaluated in FP32 (fast
    // intrinsics, this translation unit): the initial C/O/e equilibrium and the start
    // state's sources cost ~2000 FP64 FMA slots per cell, 8 ms on the 128^3 slab.
    CellC<double> c;
    double T0, x20, xp0;
    load_cell(fb, li, p, c, T0, x20, xp0);
    const CellC<float> cf = cast_cell<float>(c);
    LaneState s;
    s.t = 0.0;
    s.xH2 = x20;
    s.xHp = xp0;
    ChemT<float> b0 = chem_T(cf, float(T0), p.flags);
    Equil<float> q0 = equilibrium(cf, b0, float(x20), float(xp0), -1.f);
    s.xe = double(q0.xe); s.xCp = double(q0.xCp); s.xCO = double(q0.xCO);
    s.mu = c.muH / (1.1 + s.xe - x20);
    s.Tmu = T0 / s.mu;
    float td = -1.f;
    double H0, CH2, CHp;
    start_sources<float>(cf, p, s, td, H0, CH2, CHp);
    // r = dt / dts_1 without the cap at dt: the predicted substep count above 1, and
    // below 1 how far the state moves within its single substep (more Newton iterations
    // the closer r is to 1: 3.0 at r ~ 2^-10, 4.1 at r ~ 2^-1 on the slab).  Classes are
    // quarter octaves of r from 2^-16 to 2^16.
    const double e = c.K * s.Tmu;
    double r = 0.0;
    if (fabs(H0) > 0.0) r = fmax(r, fabs(H0) * dt / (p.limiter * e));
    r = fmax(r, fabs(CH2) * dt / p.limiter);
    r = fmax(r, fabs(CHp) * dt / p.limiter);
    int b = ORDER_BUCKETS - 1;  // unknown cost (non-finite): schedule first
    if (isfinite(r)) {
      const double l = (r > 0.0) ? log2(r) : -1e30;
      const double u = 4.0 * (l + 16.0);
      b = (u <= 0.0) ? 0 : (u >= ORDER_BUCKETS - 1 ? ORDER_BUCKETS - 1 : (int)u);
    }
    const int k = ORDER_BUCKETS - 1 - b;  // ascending key = decreasing cost
    key[gi] = (unsigned char)k;
    atomicAdd(&sh[k], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

__global__ void k_order_scan(unsigned* hist) {
  // one warp: exclusive scan of ORDER_BUCKETS counts, 4 per lane
  const int lane = threadIdx.x;
  unsigned v[ORDER_BUCKETS / 32];
  unsigned loc = 0;
  for (int j = 0; j < ORDER_BUCKETS / 32; ++j) {
    v[j] = hist[lane * (ORDER_BUCKETS / 32) + j];
    loc += v[j];
  }
  unsigned inc = loc;
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += t;
  }
  unsigned run = inc - loc;
  for (int j = 0; j < ORDER_BUCKETS / 32; ++j) {
    hist[lane * (ORDER_BUCKETS / 32) + j] = run;
    run += v[j];
  }
}

__global__ void __launch_bounds__(256) k_order_scatter(const unsigned char* __restrict__ key, long long ntotal,
                                                       unsigned* __restrict__ offs, unsigned* __restrict__ order) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  // every lane of a warp walks the same number of trips, so the warp-wide match and
  // shuffles below always see all 32 lanes
  const long long base0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31);
  for (long long w0 = base0; w0 < ntotal; w0 += stride) {
    const long long gi = w0 + (threadIdx.x & 31);
    const bool live = gi < ntotal;
    const unsigned k = live ? (unsigned)key[gi] : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    unsigned pos = 0;
    if (live && lane == leader) pos = atomicAdd(&offs[k], (unsigned)__popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (live) order[pos + __popc(peers & ((1u << lane) - 1u))] = (unsigned)gi;
  }
}

// One thread per cell: the step's prologue (initial C/O/e equilibrium, mu, T_mu) and
// its start-state sources in FP64, as the step kernel computes them.
__global__ void __launch_bounds__(128) k_rates(DevFields f, DevParams p, double dt, long long ntotal,
                                               double* __restrict__ rate, double* __restrict__ dts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ntotal;
       i += (long long)gridDim.x * blockDim.x) {
    CellC<double> c;
    double T0, x20, xp0;
    load_cell(f, i, p, c, T0, x20, xp0);
    LaneState s;
    s.t = 0.0;
    s.xH2 = x20;
    s.xHp = xp0;
    ChemT<double> b0 = chem_T(c, T0, p.flags);
    Equil<double> q0 = equilibrium(c, b0, x20, xp0, -1.0);
    s.xe = q0.xe; s.xCp = q0.xCp; s.xCO = q0.xCO;
    s.mu = c.muH / (1.1 + s.xe - x20);
    s.Tmu = T0 / s.mu;
    double td = -1.0, H0, CH2, CHp;
    start_sources<double>(c, p, s, td, H0, CH2, CHp);
    if (rate) {
      rate[3 * i + 0] = CH2;
      rate[3 * i + 1] = CHp;
      rate[3 * i + 2] = H0 / (c.K * s.Tmu);
    }
    if (dts) {
      bool last;
      dts[i] = substep_len(p, dt, c.K * s.Tmu, H0, CH2, CHp, last);
    }
  }
}

}  // namespace

cudaError_t launch_rates(const DevFields& f, const DevParams& p, double dt, long long ntotal, double* rate,
                         double* dts, int num_sms, cudaStream_t st) {
  long long nb = (ntotal + 127) / 128;
  const long long cap = (long long)num_sms * 8;
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  DevParams q = p;
  q.order = nullptr;
  k_rates<<<(int)nb, 128, 0, st>>>(f, q, dt, ntotal, rate, dts);
  return cudaGetLastError();
}

cudaError_t launch_order(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         long long ntotal, unsigned char* key, unsigned* hist, unsigned* order, int num_sms,
                         cudaStream_t st) {
  if (cudaMemsetAsync(hist, 0, ORDER_BUCKETS * sizeof(unsigned), st) != cudaSuccess) return cudaGetLastError();
  long long nb = (ntotal + 127) / 128;
  const long long cap = (long long)num_sms * 8;
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  DevParams q = p;
  q.order = nullptr;
  if (batch) k_order_key<true><<<(int)nb, 128, 0, st>>>(f, d_boxes, q, dt, ntotal, key, hist);
  else k_order_key<false><<<(int)nb, 128, 0, st>>>(f, d_boxes, q, dt, ntotal, key, hist);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_order_scan<<<1, 32, 0, st>>>(hist);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  long long ns = (ntotal + 255) / 256;
  if (ns > (long long)num_sms * 16) ns = (long long)num_sms * 16;
  if (ns < 1) ns = 1;
  k_order_scatter<<<(int)ns, 256, 0, st>>>(key, ntotal, hist, order);
  return cudaGetLastError();
}

}  // namespace tcg
