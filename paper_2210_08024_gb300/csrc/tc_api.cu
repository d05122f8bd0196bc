// C ABI of the thermochemistry library (declared in include/tc.h).
//
// Owns the handle: parameters, a small device workspace (the work-queue cursor, a
// status counter, the batched box table), reusable device buffers for the host-buffer
// entry point, and the CUDA graph of the batched launch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "../../include/tc.h"
#include "../../include/tc_onezone.h"
#include "../../include/tc_pdr.h"
#include "../../include/tc_peak.h"
#include "tc_launch.h"
#include "tc_mlp_mma.cuh"
#include "tc_onezone.cuh"
#include "tc_order.cuh"
#include "tc_pdr.cuh"

namespace tcg {
int occupancy_mode0_impl(int block);
int occupancy_mode1_impl(int block);
int occupancy_mode2_impl(int block);
int occupancy_mode3_impl(int block);
int occupancy_mode4_impl(int block);
}  // namespace tcg

constexpr int TUNE_CLASSES = 48;

static int size_class(long long n) {
  int c = 0;
  while (n > 1 && c < TUNE_CLASSES - 1) {
    n >>= 1;
    ++c;
  }
  return c;
}

struct tc_handle {
  tc_params p;
  int device = 0;
  int num_sms = 0;
  unsigned long long* d_cursor = nullptr;  // work-queue cursor (8 B)
  unsigned long long* d_count = nullptr;   // status reduction counter (8 B)
  tcg::BoxTable* d_boxes = nullptr;        // batched launch box table
  tcg::BoxTable* h_boxes = nullptr;        // pinned host copy (graph memcpy source)
  long long launches = 0;
  // host-buffer entry point scratch
  double* d_buf = nullptr;
  size_t d_buf_cells = 0;
  int* d_ibuf = nullptr;
  // batched graph cache: the executable graph, what it was captured for (box table,
  // dt, parameters, stream; compared in full, not by a hash), and an event recorded
  // after each of its launches (the pinned h_boxes and d_boxes are reused only after
  // the last launch has finished with them)
  cudaGraphExec_t gexec = nullptr;
  tcg::BoxTable gtb;
  double gdt = 0.0;
  tc_params gp;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gdone = nullptr;
  // MLP seed weights (device) -- loaded by tc_load_mlp -- and their tensor-core layout
  void* d_mlp = nullptr;
  tcg::MlpMma* d_mlp_mma = nullptr;
  size_t mlp_bytes = 0;
  // cost-ordered work queue (tc_params.order_cells): class keys, histogram, order
  unsigned char* d_okey = nullptr;
  unsigned* d_ohist = nullptr;
  unsigned* d_order = nullptr;
  size_t order_cells = 0;
  // launch shapes recorded by tc_autotune, by size class floor(log2(ncell))
  struct Tuned {
    int valid, block, blocks_per_sm, lanes_per_cell;
  } tuned[TUNE_CLASSES] = {};
  // driver workspace (tc_eq_curves, tc_pdr): per-cell arrays and the parameter arrays
  double* d_eq = nullptr;
  int* d_eqi = nullptr;
  size_t eq_cells = 0;
  double* d_eqpar = nullptr;
  size_t eqpar_len = 0;
};

// The step kernel's warp-level tensor-core inference of the seed network on rows of
// raw features (tc_seed_predict): each warp takes 32 rows at a time, all its lanes
// together; rows past B are zero features whose outputs are dropped.
namespace {
__global__ void __launch_bounds__(128) k_seed_predict(const tcg::MlpMma* __restrict__ m, const float* __restrict__ X,
                                                      int B, float* __restrict__ out) {
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (long long base = warp * 32; base < B; base += nw * 32) {
    const long long r = base + lane;
    float f[tcg::MLP_IN], o[tcg::MLP_OUT];
    for (int k = 0; k < tcg::MLP_IN; ++k) f[k] = (r < B) ? X[r * tcg::MLP_IN + k] : 0.f;
    tcg::mlp_infer_warp(m, f, o);
    if (r < B)
      for (int j = 0; j < tcg::MLP_OUT; ++j) out[r * tcg::MLP_OUT + j] = o[j];
  }
}
}  // namespace

extern "C" {

const char* tc_strerror(int code) {
  switch (code) {
    case TC_OK: return "ok";
    case TC_EINVAL: return "invalid argument";
    case TC_ECUDA: return "CUDA runtime error";
    case TC_ENOMEM: return "out of memory";
    case TC_ENOMLP: return "seeded mode requested before tc_load_mlp";
    case TC_ENODEV: return "no sm_103 CUDA device";
    default: return "unknown error";
  }
}

int tc_params_default(tc_params* p, int mode) {
  if (!p) return TC_EINVAL;
  memset(p, 0, sizeof(*p));
  p->dvdr_kms_pc = 1.0;
  p->T_cmb = 2.73;
  p->chi0 = 1.0;
  p->opt_over_fuv = 1.0;
  p->tau_opt_over_tau_pe = 1.0 / 3.0;
  p->limiter = 0.1;
  p->fd_rel_step = 1e-3;
  p->newton_rtol = 1e-12;
  p->T_floor = 1.0;
  p->newton_max = 50;
  p->max_substeps = 1000000;
  p->mode = mode;
  p->flags = 0;
  p->newton_rtol_mixed = 1e-6;
  p->block = 0;
  p->blocks_per_sm = 0;
  p->order_cells = 1;
  return TC_OK;
}

static bool mode_ok(int m) { return m >= TC_MODE_PAPER_FP64 && m <= TC_MODE_NEWTON_FP64_SEEDED; }

int tc_create(const tc_params* p, tc_handle** out) {
  if (!p || !out || !mode_ok(p->mode)) return TC_EINVAL;
  if (!(p->limiter > 0.0) || !(p->fd_rel_step > 0.0) || p->newton_max < 1 || p->max_substeps < 1) return TC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TC_ENODEV;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return TC_ECUDA;
  if (prop.major < 10) return TC_ENODEV;
  tc_handle* h = new (std::nothrow) tc_handle();
  if (!h) return TC_ENOMEM;
  h->p = *p;
  h->device = dev;
  h->num_sms = prop.multiProcessorCount;
  if (cudaMalloc(&h->d_cursor, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    delete h;
    return TC_ENOMEM;
  }
  h->d_count = h->d_cursor + 1;
  *out = h;
  return TC_OK;
}

void tc_destroy(tc_handle* h) {
  if (!h) return;
  if (h->gdone) {
    cudaEventSynchronize(h->gdone);
    cudaEventDestroy(h->gdone);
  }
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  cudaFree(h->d_cursor);
  cudaFree(h->d_boxes);
  cudaFreeHost(h->h_boxes);
  cudaFree(h->d_buf);
  cudaFree(h->d_ibuf);
  cudaFree(h->d_mlp);
  cudaFree(h->d_mlp_mma);
  cudaFree(h->d_eq);
  cudaFree(h->d_eqi);
  cudaFree(h->d_eqpar);
  cudaFree(h->d_okey);
  cudaFree(h->d_ohist);
  cudaFree(h->d_order);
  delete h;
}

long long tc_launch_count(const tc_handle* h) { return h ? h->launches : -1; }

static tcg::DevParams dev_params(const tc_params& p) {
  tcg::DevParams d;
  d.dvdr_kms_pc = p.dvdr_kms_pc;
  d.T_cmb = p.T_cmb;
  d.chi0 = p.chi0;
  d.opt_over_fuv = p.opt_over_fuv;
  d.tau_ratio = p.tau_opt_over_tau_pe;
  d.limiter = p.limiter;
  d.fd_rel = p.fd_rel_step;
  d.rtol = p.newton_rtol;
  d.rtol_mixed = p.newton_rtol_mixed;
  d.T_floor = p.T_floor;
  d.newton_max = p.newton_max;
  d.max_sub = p.max_substeps;
  d.flags = p.flags;
  return d;
}

static bool aligned8(const void* q) { return (((uintptr_t)q) & 7u) == 0; }

static int check_fields(const tc_fields* f) {
  if (!f || f->ncell < 0) return TC_EINVAL;
  if (f->ncell == 0) return TC_OK;
  const void* req[] = {f->n, f->chi_pe, f->chi_lw, f->f_shld_h2, f->xi_cr, f->T, f->x_h2, f->x_hp};
  for (const void* q : req)
    if (!q || !aligned8(q)) return TC_EINVAL;
  const void* opt[] = {f->f_shld_c, f->F_lyc, f->Zg, f->Zd, f->x_e, f->x_cp, f->x_co};
  for (const void* q : opt)
    if (q && !aligned8(q)) return TC_EINVAL;
  if (f->cost_hint && (((uintptr_t)f->cost_hint) & 3u)) return TC_EINVAL;
  if (!f->Zg && !(f->Zg_val >= 0.0)) return TC_EINVAL;
  if (!f->Zd && !(f->Zd_val >= 0.0)) return TC_EINVAL;
  return TC_OK;
}

static tcg::DevFields dev_fields(const tc_fields* f) {
  tcg::DevFields d;
  d.n = f->n; d.chi_pe = f->chi_pe; d.chi_lw = f->chi_lw; d.fh2 = f->f_shld_h2; d.fc = f->f_shld_c;
  d.Flyc = f->F_lyc; d.xi = f->xi_cr; d.Zg = f->Zg; d.Zd = f->Zd;
  d.T = f->T; d.xH2 = f->x_h2; d.xHp = f->x_hp; d.xe = f->x_e; d.xCp = f->x_cp; d.xCO = f->x_co;
  d.nsub = f->nsub; d.status = f->status; d.iters = f->newton_iters;
  d.hint = f->cost_hint;
  d.ncell = f->ncell;
  d.Zg_val = f->Zg_val; d.Zd_val = f->Zd_val;
  return d;
}

int tc_df64_source_check(const tc_params* p, const tc_fields* f, double* err, void* stream) {
  if (!p || !err) return TC_EINVAL;
  const int rc = check_fields(f);
  if (rc != TC_OK || f->ncell == 0) return rc;
  if (!aligned8(err)) return TC_EINVAL;
  return tcg::launch_df64_source_check(dev_fields(f), dev_params(*p), err, (cudaStream_t)stream) == cudaSuccess
             ? TC_OK
             : TC_ECUDA;
}

static int kernel_mode(int mode) {
  switch (mode) {
    case TC_MODE_PAPER_FP64: return 0;
    case TC_MODE_NEWTON_FP64: return 1;
    case TC_MODE_MIXED: return 2;
    case TC_MODE_MIXED_SEEDED: return 3;
    default: return 4;  // TC_MODE_NEWTON_FP64_SEEDED
  }
}

static int coop_occupancy(int kmode, int block) {
  return (kmode == 1) ? tcg::occupancy_mode1_coop(block) : tcg::occupancy_mode2_coop(block);
}

// Launch shape of one step launch: threads per block, grid and lanes per cell.  Explicit
// tc_params values win; otherwise the shape tc_autotune recorded for the launch's size
// class; otherwise 128 threads, the occupancy limit, and for modes 1 and 2 four lanes per
// cell when every cell's four lanes fit the cooperative kernel's resident lanes at once
// (4096 random states: FP64 Newton 73.1 ms against 108.8 ms with one lane, mixed 43.7
// against 55.7 ms; the mixed solve builds one FP32 Jacobian per solve and spends most of
// its time in the df64 polish and substep-start sources, which four lanes do not
// shorten).  The persistent grid never exceeds the blocks that hold one lane per cell
// lane.
struct Shape {
  int grid, block, lpc;
};
static Shape launch_shape(tc_handle* h, int kmode, bool batch, long long ntotal) {
  int b = h->p.block, per_sm = h->p.blocks_per_sm, lpc = h->p.lanes_per_cell;
  const bool coop_ok = (kmode == 1 || kmode == 2) && !batch;
  const tc_handle::Tuned& t = h->tuned[size_class(ntotal)];
  if (t.valid && !batch && b <= 0 && per_sm <= 0 && lpc <= 0) {
    b = t.block;
    per_sm = t.blocks_per_sm;
    lpc = t.lanes_per_cell;
  }
  if (b <= 0) b = 128;
  if (b > 128) b = 128;  // kernels are compiled with __launch_bounds__(128)
  b = (b / 32) * 32;
  if (b < 32) b = 32;
  if (!coop_ok) lpc = 1;
  if (lpc <= 0) lpc = (coop_ok && ntotal * 4 <= (long long)h->num_sms * coop_occupancy(kmode, b) * b) ? 4 : 1;
  if (lpc != 4) lpc = 1;
  if (per_sm <= 0) {
    per_sm = (lpc == 4) ? coop_occupancy(kmode, b)
             : (kmode == 0) ? tcg::occupancy_mode0_impl(b)
             : (kmode == 1) ? tcg::occupancy_mode1_impl(b)
             : (kmode == 2) ? tcg::occupancy_mode2_impl(b)
             : (kmode == 3) ? tcg::occupancy_mode3_impl(b) : tcg::occupancy_mode4_impl(b);
  }
  long long g = (long long)h->num_sms * per_sm;
  long long need = (ntotal * lpc + b - 1) / b;
  if (g > need) g = need;
  if (g < 1) g = 1;
  return Shape{(int)g, b, lpc};
}

// Grows the cost-ordering workspace to ncell cells (not while `st` is being captured).
// Returns false if there is none to use.
static bool order_workspace(tc_handle* h, long long ncell, cudaStream_t st) {
  if (ncell > 4000000000LL) return false;
  if (h->order_cells >= (size_t)ncell && h->d_order) return true;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
  if (h->gexec) {  // the cached batched graph points at the old workspace
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  cudaFree(h->d_okey);
  cudaFree(h->d_order);
  h->d_okey = nullptr;
  h->d_order = nullptr;
  h->order_cells = 0;
  if (!h->d_ohist && cudaMalloc(&h->d_ohist, tcg::ORDER_BUCKETS * sizeof(unsigned)) != cudaSuccess) return false;
  if (cudaMalloc(&h->d_okey, (size_t)ncell) != cudaSuccess) return false;
  if (cudaMalloc(&h->d_order, (size_t)ncell * sizeof(unsigned)) != cudaSuccess) {
    cudaFree(h->d_okey);
    h->d_okey = nullptr;
    return false;
  }
  h->order_cells = (size_t)ncell;
  return true;
}

static int enqueue(tc_handle* h, bool batch, const tcg::DevFields& f, long long ntotal, double dt, cudaStream_t st) {
  int kmode = kernel_mode(h->p.mode);
  if (h->p.mode == TC_MODE_MIXED_SEEDED || h->p.mode == TC_MODE_NEWTON_FP64_SEEDED) {
    if (!h->d_mlp) return TC_ENOMLP;
  }
  const Shape sh = launch_shape(h, kmode, batch, ntotal);
  const int grid = sh.grid, block = sh.block;
  if (cudaMemsetAsync(h->d_cursor, 0, sizeof(unsigned long long), st) != cudaSuccess) return TC_ECUDA;
  tcg::DevParams dp = dev_params(h->p);
  dp.mlp_mma = h->d_mlp_mma;
  // cost-ordered queue: only worth it when the launch holds more cells than a few warps
  if (h->p.order_cells && ntotal > 256 && order_workspace(h, ntotal, st)) {
    if (tcg::launch_order(batch, f, h->d_boxes, dp, dt, ntotal, h->d_okey, h->d_ohist, h->d_order, h->num_sms, st) !=
        cudaSuccess)
      return TC_ECUDA;
    h->launches += 3;
    dp.order = h->d_order;
  }
  cudaError_t e;
  if (sh.lpc == 4 && kmode == 1) e = tcg::launch_mode1_coop(f, dp, dt, h->d_cursor, ntotal, grid, block, st);
  else if (sh.lpc == 4 && kmode == 2) e = tcg::launch_mode2_coop(f, dp, dt, h->d_cursor, ntotal, grid, block, st);
  else if (kmode == 0) e = tcg::launch_mode0(batch, f, h->d_boxes, dp, dt, h->d_cursor, ntotal, grid, block, st);
  else if (kmode == 1) e = tcg::launch_mode1(batch, f, h->d_boxes, dp, dt, h->d_cursor, ntotal, grid, block, st);
  else if (kmode == 2) e = tcg::launch_mode2(batch, f, h->d_boxes, dp, dt, h->d_cursor, ntotal, grid, block, st);
  else if (kmode == 3)
    e = tcg::launch_mode3(batch, f, h->d_boxes, dp, dt, h->d_cursor, ntotal, grid, block, st,
                          (const tcg::MlpDev*)h->d_mlp);
  else
    e = tcg::launch_mode4(batch, f, h->d_boxes, dp, dt, h->d_cursor, ntotal, grid, block, st,
                          (const tcg::MlpDev*)h->d_mlp);
  if (e != cudaSuccess) return TC_ECUDA;
  h->launches += 1;
  return TC_OK;
}

int tc_step(tc_handle* h, const tc_fields* f, double dt_s, void* stream) {
  if (!h) return TC_EINVAL;
  int rc = check_fields(f);
  if (rc != TC_OK) return rc;
  if (!(dt_s >= 0.0) || !isfinite(dt_s)) return TC_EINVAL;
  if (f->ncell == 0) return TC_OK;
  return enqueue(h, false, dev_fields(f), f->ncell, dt_s, (cudaStream_t)stream);
}

int tc_rates(tc_handle* h, const tc_fields* f, double dt_s, double* rate, double* dts, void* stream) {
  if (!h) return TC_EINVAL;
  int rc = check_fields(f);
  if (rc != TC_OK) return rc;
  if (!(dt_s >= 0.0) || !isfinite(dt_s)) return TC_EINVAL;
  if (f->ncell == 0 || (!rate && !dts)) return TC_OK;
  if (tcg::launch_rates(dev_fields(f), dev_params(h->p), dt_s, f->ncell, rate, dts, h->num_sms,
                        (cudaStream_t)stream) != cudaSuccess)
    return TC_ECUDA;
  h->launches += 1;
  return TC_OK;
}

int tc_autotune(tc_handle* h, const tc_fields* f, double dt_s, void* stream, tc_tune_choice* best) {
  if (!h || !best) return TC_EINVAL;
  int rc = check_fields(f);
  if (rc != TC_OK) return rc;
  if (f->ncell < 1 || !(dt_s >= 0.0) || !isfinite(dt_s)) return TC_EINVAL;
  const int kmode = kernel_mode(h->p.mode);
  if ((kmode == 3 || kmode == 4) && !h->d_mlp) return TC_ENOMLP;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)f->ncell;
  // Candidates run on a scratch copy of the state; the inputs are only read.
  double* scratch = nullptr;
  if (cudaMalloc(&scratch, 3 * n * sizeof(double)) != cudaSuccess) return TC_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaFree(scratch);
    return TC_ECUDA;
  }
  tc_fields d = *f;
  d.T = scratch;
  d.x_h2 = scratch + n;
  d.x_hp = scratch + 2 * n;
  d.x_e = d.x_cp = d.x_co = nullptr;
  d.nsub = d.status = d.newton_iters = nullptr;
  const tc_params saved = h->p;
  const tc_handle::Tuned told = h->tuned[size_class(f->ncell)];
  h->tuned[size_class(f->ncell)].valid = 0;
  // four lanes per cell only where the cooperative kernel holds the launch's cells in at
  // most 8 waves of resident lanes (beyond that it is slower by construction)
  const bool coop_ok = (kmode == 1 || kmode == 2) &&
                       (long long)f->ncell * 4 <= 8LL * h->num_sms * coop_occupancy(kmode, 128) * 128;
  const int blocks[3] = {32, 64, 128};
  const int per_sms[2] = {0, 4};
  const int lpcs[2] = {1, 4};
  // One run in the default shape first (it also sets how often each candidate repeats).
  auto run = [&](float* ms) -> int {
    const double* src[3] = {f->T, f->x_h2, f->x_hp};
    for (int k = 0; k < 3; ++k)
      if (cudaMemcpyAsync(scratch + k * n, src[k], n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return TC_ECUDA;
    if (cudaEventRecord(e0, st) != cudaSuccess) return TC_ECUDA;
    const int r = enqueue(h, false, dev_fields(&d), f->ncell, dt_s, st);
    if (r != TC_OK) return r;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return TC_ECUDA;
    return (cudaEventElapsedTime(ms, e0, e1) == cudaSuccess) ? TC_OK : TC_ECUDA;
  };
  float ms0 = 0.f;
  h->p.block = 0;
  h->p.blocks_per_sm = 0;
  h->p.lanes_per_cell = 0;
  rc = run(&ms0);
  const int reps = (rc == TC_OK && ms0 < 20.f) ? 3 : 1;
  tc_tune_choice bestc = {0, 0, 0, 3.4e38f};
  for (int ib = 0; ib < 3 && rc == TC_OK; ++ib)
    for (int ip = 0; ip < 2 && rc == TC_OK; ++ip)
      for (int il = 0; il < (coop_ok ? 2 : 1) && rc == TC_OK; ++il) {
        h->p.block = blocks[ib];
        h->p.blocks_per_sm = per_sms[ip];
        h->p.lanes_per_cell = lpcs[il];
        float tmin = 3.4e38f;
        for (int r = 0; r < reps && rc == TC_OK; ++r) {
          float ms = 0.f;
          rc = run(&ms);
          if (ms < tmin) tmin = ms;
        }
        if (rc == TC_OK && tmin < bestc.ms) bestc = tc_tune_choice{blocks[ib], per_sms[ip], lpcs[il], tmin};
      }
  h->p = saved;
  if (rc == TC_OK) {
    h->tuned[size_class(f->ncell)] = tc_handle::Tuned{1, bestc.block, bestc.blocks_per_sm, bestc.lanes_per_cell};
    *best = bestc;
  } else {
    h->tuned[size_class(f->ncell)] = told;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  return rc;
}

int tc_step_host(tc_handle* h, const tc_fields* f, double dt_s, void* stream) {
  if (!h) return TC_EINVAL;
  int rc = check_fields(f);
  if (rc != TC_OK) return rc;
  if (!(dt_s >= 0.0) || !isfinite(dt_s)) return TC_EINVAL;
  if (f->ncell == 0) return TC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)f->ncell;
  const int NIN = 9, NST = 6;
  if (h->d_buf_cells < n) {
    cudaFree(h->d_buf);
    cudaFree(h->d_ibuf);
    h->d_buf = nullptr;
    h->d_ibuf = nullptr;
    h->d_buf_cells = 0;
    if (cudaMalloc(&h->d_buf, n * sizeof(double) * (NIN + NST)) != cudaSuccess) return TC_ENOMEM;
    if (cudaMalloc(&h->d_ibuf, n * sizeof(int) * 3) != cudaSuccess) return TC_ENOMEM;
    h->d_buf_cells = n;
  }
  double* b = h->d_buf;
  const double* hin[NIN] = {f->n, f->chi_pe, f->chi_lw, f->f_shld_h2, f->f_shld_c, f->F_lyc, f->xi_cr, f->Zg, f->Zd};
  double* din[NIN];
  for (int k = 0; k < NIN; ++k) {
    din[k] = hin[k] ? b + (size_t)k * n : nullptr;
    if (hin[k] && cudaMemcpyAsync(din[k], hin[k], n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return TC_ECUDA;
  }
  double* hst[NST] = {f->T, f->x_h2, f->x_hp, f->x_e, f->x_cp, f->x_co};
  double* dst[NST];
  for (int k = 0; k < NST; ++k) {
    dst[k] = hst[k] ? b + (size_t)(NIN + k) * n : nullptr;
    if (k < 3 && cudaMemcpyAsync(dst[k], hst[k], n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return TC_ECUDA;
  }
  tc_fields d = *f;
  d.n = din[0]; d.chi_pe = din[1]; d.chi_lw = din[2]; d.f_shld_h2 = din[3]; d.f_shld_c = din[4]; d.F_lyc = din[5];
  d.xi_cr = din[6]; d.Zg = din[7]; d.Zd = din[8];
  d.T = dst[0]; d.x_h2 = dst[1]; d.x_hp = dst[2]; d.x_e = dst[3]; d.x_cp = dst[4]; d.x_co = dst[5];
  d.nsub = f->nsub ? h->d_ibuf : nullptr;
  d.status = f->status ? h->d_ibuf + n : nullptr;
  d.newton_iters = f->newton_iters ? h->d_ibuf + 2 * n : nullptr;
  d.cost_hint = nullptr;  // a host array here; the predicted order is used
  rc = enqueue(h, false, dev_fields(&d), f->ncell, dt_s, st);
  if (rc != TC_OK) return rc;
  for (int k = 0; k < NST; ++k)
    if (hst[k] && cudaMemcpyAsync(hst[k], dst[k], n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return TC_ECUDA;
  if (f->nsub && cudaMemcpyAsync(f->nsub, d.nsub, n * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TC_ECUDA;
  if (f->status && cudaMemcpyAsync(f->status, d.status, n * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TC_ECUDA;
  if (f->newton_iters &&
      cudaMemcpyAsync(f->newton_iters, d.newton_iters, n * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TC_ECUDA;
  return TC_OK;
}

int tc_step_batch(tc_handle* h, const tc_fields* boxes, int nbox, double dt_s, void* stream) {
  if (!h || !boxes || nbox < 1 || nbox > tcg::MAX_BOX) return TC_EINVAL;
  if (!(dt_s >= 0.0) || !isfinite(dt_s)) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!h->d_boxes) {
    if (cudaMalloc(&h->d_boxes, sizeof(tcg::BoxTable)) != cudaSuccess) return TC_ENOMEM;
    if (cudaMallocHost(&h->h_boxes, sizeof(tcg::BoxTable)) != cudaSuccess) return TC_ENOMEM;
  }
  tcg::BoxTable tb;
  memset(&tb, 0, sizeof(tb));
  tb.nbox = nbox;
  long long tot = 0;
  for (int b = 0; b < nbox; ++b) {
    int rc = check_fields(&boxes[b]);
    if (rc != TC_OK) return rc;
    tb.start[b] = tot;
    tb.box[b] = dev_fields(&boxes[b]);
    tot += boxes[b].ncell;
  }
  tb.start[nbox] = tot;
  if (tot == 0) return TC_OK;
  const bool same = h->gexec && memcmp(&tb, &h->gtb, sizeof(tb)) == 0 && memcmp(&dt_s, &h->gdt, sizeof(dt_s)) == 0 &&
                    memcmp(&h->p, &h->gp, sizeof(h->p)) == 0 && st == h->gstream;
  if (!same) {
    // The previous graph's launch may still be in flight, reading h_boxes (its memcpy
    // node) and d_boxes (its kernel): wait for it before either is rewritten.
    if (h->gdone && cudaEventSynchronize(h->gdone) != cudaSuccess) return TC_ECUDA;
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    memcpy(h->h_boxes, &tb, sizeof(tb));
    if (h->p.order_cells) order_workspace(h, tot, st);  // allocate before the capture
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return TC_ECUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaStreamDestroy(cap);
      return TC_ECUDA;
    }
    cudaError_t e = cudaMemcpyAsync(h->d_boxes, h->h_boxes, sizeof(tcg::BoxTable), cudaMemcpyHostToDevice, cap);
    long long before = h->launches;
    int rc = (e == cudaSuccess) ? enqueue(h, true, tb.box[0], tot, dt_s, cap) : TC_ECUDA;
    h->launches = before;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc != TC_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e2 != cudaSuccess) return TC_ECUDA;
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return TC_ECUDA;
    memcpy(&h->gtb, &tb, sizeof(tb));
    memcpy(&h->gdt, &dt_s, sizeof(dt_s));
    memcpy(&h->gp, &h->p, sizeof(h->p));
    h->gstream = st;
  }
  if (!h->gdone && cudaEventCreateWithFlags(&h->gdone, cudaEventDisableTiming) != cudaSuccess) return TC_ECUDA;
  if (cudaGraphLaunch(h->gexec, st) != cudaSuccess) return TC_ECUDA;
  if (cudaEventRecord(h->gdone, st) != cudaSuccess) return TC_ECUDA;
  h->launches += 1;
  return TC_OK;
}

int tc_seed_predict(tc_handle* h, const float* X, int B, float* out, void* stream) {
  if (!h || B < 0 || (B > 0 && (!X || !out))) return TC_EINVAL;
  if (!h->d_mlp_mma) return TC_ENOMLP;
  if (B == 0) return TC_OK;
  long long nb = ((long long)B + 127) / 128;
  if (nb > (long long)h->num_sms * 8) nb = (long long)h->num_sms * 8;
  k_seed_predict<<<(int)nb, 128, 0, (cudaStream_t)stream>>>(h->d_mlp_mma, X, B, out);
  if (cudaGetLastError() != cudaSuccess) return TC_ECUDA;
  h->launches += 1;
  return TC_OK;
}

int tc_load_mlp(tc_handle* h, const void* blob, size_t bytes) {
  if (!h || !blob || bytes != sizeof(tcg::MlpDev)) return TC_EINVAL;
  const tcg::MlpDev* hb = (const tcg::MlpDev*)blob;
  if (hb->magic != tcg::MLP_MAGIC || hb->version != tcg::MLP_VERSION || hb->bytes != sizeof(tcg::MlpDev) ||
      hb->n_in != (uint32_t)tcg::MLP_IN || hb->n_hid != (uint32_t)tcg::MLP_HID || hb->n_out != (uint32_t)tcg::MLP_OUT)
    return TC_EINVAL;
  cudaFree(h->d_mlp);
  cudaFree(h->d_mlp_mma);
  h->d_mlp = nullptr;
  h->d_mlp_mma = nullptr;
  h->mlp_bytes = 0;
  if (cudaMalloc(&h->d_mlp, bytes) != cudaSuccess) return TC_ENOMEM;
  if (cudaMalloc(&h->d_mlp_mma, sizeof(tcg::MlpMma)) != cudaSuccess) return TC_ENOMEM;
  if (cudaMemcpy(h->d_mlp, blob, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return TC_ECUDA;
  if (tcg::mlp_mma_layout((const tcg::MlpDev*)h->d_mlp, h->d_mlp_mma, 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return TC_ECUDA;
  h->mlp_bytes = bytes;
  return TC_OK;
}

}  // extern "C"

// ----- status reduction
namespace {
__global__ void k_count_bad(const int* __restrict__ status, long long n, unsigned long long* count) {
  unsigned long long local = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    local += ((status[i] & TC_ST_ERROR_MASK) != 0);
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}
}  // namespace

extern "C" int tc_sync_status(tc_handle* h, const int* status, long long ncell, void* stream, long long* nbad) {
  if (!h || !nbad || ncell < 0 || (ncell > 0 && !status)) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(h->d_count, 0, sizeof(unsigned long long), st) != cudaSuccess) return TC_ECUDA;
  if (ncell > 0) {
    int grid = h->num_sms * 4;
    k_count_bad<<<grid, 256, 0, st>>>(status, ncell, h->d_count);
    if (cudaGetLastError() != cudaSuccess) return TC_ECUDA;
    h->launches += 1;
  }
  unsigned long long v = 0;
  if (cudaMemcpyAsync(&v, h->d_count, sizeof(v), cudaMemcpyDeviceToHost, st) != cudaSuccess) return TC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TC_ECUDA;
  *nbad = (long long)v;
  return TC_OK;
}

// ----- driver workspace shared by the one-zone and PDR drivers
// Grows the per-cell workspace (DRIVER_NW doubles and DRIVER_NI ints per cell) and the
// parameter buffer, waits for earlier work on the stream (it may still read the previous
// call's parameters), copies the five host parameter arrays and waits for the copies.
static const size_t DRIVER_NW = 11;
// ints: the latest launch's status, the OR of the earlier ones, and each cell's Newton
// iterations in the latest chunk (the cost hint of the next chunk's cell order)
static const size_t DRIVER_NI = 3;

static int driver_setup(tc_handle* h, size_t ncell, const double* const hp[5], const size_t len[5], double* dp[5],
                        cudaStream_t st) {
  if (h->eq_cells < ncell) {
    cudaFree(h->d_eq);
    cudaFree(h->d_eqi);
    h->d_eq = nullptr;
    h->d_eqi = nullptr;
    h->eq_cells = 0;
    if (cudaMalloc(&h->d_eq, ncell * DRIVER_NW * sizeof(double)) != cudaSuccess) return TC_ENOMEM;
    if (cudaMalloc(&h->d_eqi, ncell * DRIVER_NI * sizeof(int)) != cudaSuccess) return TC_ENOMEM;
    h->eq_cells = ncell;
  }
  size_t npar = 0;
  for (int k = 0; k < 5; ++k) npar += len[k];
  if (h->eqpar_len < npar) {
    cudaFree(h->d_eqpar);
    h->d_eqpar = nullptr;
    h->eqpar_len = 0;
    if (cudaMalloc(&h->d_eqpar, npar * sizeof(double)) != cudaSuccess) return TC_ENOMEM;
    h->eqpar_len = npar;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return TC_ECUDA;
  size_t off = 0;
  for (int k = 0; k < 5; ++k) {
    dp[k] = h->d_eqpar + off;
    if (cudaMemcpyAsync(dp[k], hp[k], len[k] * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return TC_ECUDA;
    off += len[k];
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return TC_ECUDA;
  return TC_OK;
}

static bool all_finite_nonneg(const double* a, long long n, bool positive) {
  for (long long i = 0; i < n; ++i)
    if (!isfinite(a[i]) || a[i] < 0.0 || (positive && !(a[i] > 0.0))) return false;
  return true;
}

static bool start_state_ok(double T, double x2, double xp) {
  return T > 0.0 && isfinite(T) && x2 >= 0.0 && xp >= 0.0 && 2.0 * x2 + xp <= 1.0;
}

// Step inputs of a driver run, laid out in the workspace.
static tcg::DevFields driver_fields(tc_handle* h, size_t n, double* T, double* xH2, double* xHp, double* xe,
                                    double* xCO) {
  double* b = h->d_eq;
  tcg::DevFields f;
  memset(&f, 0, sizeof(f));
  f.n = b; f.chi_pe = b + n; f.chi_lw = b + 2 * n; f.fh2 = b + 3 * n; f.xi = b + 4 * n;
  f.Zg = b + 5 * n; f.Zd = b + 6 * n; f.chi0 = b + 7 * n;
  f.fc = nullptr; f.Flyc = nullptr;
  f.T = T; f.xH2 = xH2; f.xHp = xHp; f.xe = xe; f.xCp = nullptr; f.xCO = xCO;
  f.nsub = nullptr; f.status = h->d_eqi; f.iters = h->d_eqi + 2 * n;
  f.ncell = (long long)n;
  return f;
}

// ----- one-zone equilibrium curves (include/tc_onezone.h)
extern "C" int tc_eq_spec_default(tc_eq_spec* s) {
  if (!s) return TC_EINVAL;
  memset(s, 0, sizeof(*s));
  s->L_shld0_pc = 5.0;
  s->n_shld0 = 1e2;
  s->a_shld = 0.7;
  s->t_end_s = 1e2 * 1e6 * 3.15576e7;
  s->nchunk = 10;
  s->T_init = 3000.0;
  s->xH2_init = 0.0;
  s->xHp_init = 1e-2;
  return TC_OK;
}

extern "C" int tc_eq_curves(tc_handle* h, const tc_eq_spec* s, const tc_eq_out* o, void* stream) {
  if (!h || !s || !o) return TC_EINVAL;
  if (s->nn < 1 || s->ncurve < 1 || s->nchunk < 1 || !s->n_axis || !s->chi0 || !s->xi0 || !s->Zg || !s->Zd)
    return TC_EINVAL;
  if (!(s->t_end_s >= 0.0) || !isfinite(s->t_end_s)) return TC_EINVAL;
  if (!all_finite_nonneg(s->n_axis, s->nn, true) || !all_finite_nonneg(s->chi0, s->ncurve, false) ||
      !all_finite_nonneg(s->xi0, s->ncurve, false) || !all_finite_nonneg(s->Zg, s->ncurve, false) ||
      !all_finite_nonneg(s->Zd, s->ncurve, false))
    return TC_EINVAL;
  if (s->shielded && !(s->L_shld0_pc >= 0.0 && s->n_shld0 > 0.0 && isfinite(s->a_shld))) return TC_EINVAL;
  if (!start_state_ok(s->T_init, s->xH2_init, s->xHp_init)) return TC_EINVAL;
  const void* req[] = {o->T, o->x_h2, o->x_hp, o->x_e, o->P_k};
  for (const void* q : req)
    if (!q || !aligned8(q)) return TC_EINVAL;
  if ((o->x_co && !aligned8(o->x_co)) || (o->chg && !aligned8(o->chg))) return TC_EINVAL;
  if (h->p.mode == TC_MODE_MIXED_SEEDED || h->p.mode == TC_MODE_NEWTON_FP64_SEEDED) {
    if (!h->d_mlp) return TC_ENOMLP;
  }
  if ((double)s->nn * (double)s->ncurve > 9.0e15) return TC_EINVAL;
  const long long ncell = s->nn * (long long)s->ncurve;
  cudaStream_t st = (cudaStream_t)stream;
  const double* hp[5] = {s->n_axis, s->chi0, s->xi0, s->Zg, s->Zd};
  const size_t len[5] = {(size_t)s->nn, (size_t)s->ncurve, (size_t)s->ncurve, (size_t)s->ncurve, (size_t)s->ncurve};
  double* dp[5];
  int rc0 = driver_setup(h, (size_t)ncell, hp, len, dp, st);
  if (rc0 != TC_OK) return rc0;

  tcg::EqGrid g;
  g.n_axis = dp[0]; g.chi0 = dp[1]; g.xi0 = dp[2]; g.Zg = dp[3]; g.Zd = dp[4];
  g.nn = s->nn;
  g.ncurve = s->ncurve;
  g.shielded = s->shielded ? 1 : 0;
  g.L0_cm = s->L_shld0_pc * 3.0856775814913673e18;
  g.n0 = s->n_shld0;
  g.a = s->a_shld;
  g.T0 = s->T_init;
  g.xH20 = s->xH2_init;
  g.xHp0 = s->xHp_init;
  const size_t n = (size_t)ncell;
  tcg::DevFields f = driver_fields(h, n, o->T, o->x_h2, o->x_hp, o->x_e, o->x_co);
  tcg::EqWork w;
  w.n = const_cast<double*>(f.n); w.chi_pe = const_cast<double*>(f.chi_pe); w.chi_lw = const_cast<double*>(f.chi_lw);
  w.fh2 = const_cast<double*>(f.fh2); w.xi = const_cast<double*>(f.xi); w.Zg = const_cast<double*>(f.Zg);
  w.Zd = const_cast<double*>(f.Zd); w.chi0 = const_cast<double*>(f.chi0);
  w.prev = h->d_eq + 8 * n;
  w.st = h->d_eqi; w.st_acc = h->d_eqi + n;
  const double dt = s->t_end_s / s->nchunk;
  for (int k = 0; k < s->nchunk; ++k) {
    if (tcg::launch_eq_fields(g, w, o->T, o->x_h2, o->x_hp, k, k == s->nchunk - 1, st) != cudaSuccess)
      return TC_ECUDA;
    h->launches += 1;
    f.hint = (k > 0) ? f.iters : nullptr;  // order each chunk by the previous chunk's iterations
    int rc = enqueue(h, false, f, ncell, dt, st);
    if (rc != TC_OK) return rc;
  }
  if (tcg::launch_eq_finish(g, w, o->T, o->x_h2, o->x_hp, o->x_e, o->P_k, o->chg, o->status, st) != cudaSuccess)
    return TC_ECUDA;
  h->launches += 1;
  if (o->i_max || o->i_min) {
    if (tcg::launch_eq_extrema(g, o->P_k, o->i_max, o->i_min, st) != cudaSuccess) return TC_ECUDA;
    h->launches += 1;
  }
  return TC_OK;
}

// ----- PDR slabs (include/tc_pdr.h)
extern "C" int tc_pdr_spec_default(tc_pdr_spec* s) {
  if (!s) return TC_EINVAL;
  memset(s, 0, sizeof(*s));
  s->t_end_s = 3e2 * 1e6 * 3.15576e7;
  s->nchunk = 300;
  s->T_init = 100.0;
  s->xH2_init = 0.0;
  s->xHp_init = 1e-4;
  return TC_OK;
}

extern "C" int tc_pdr(tc_handle* h, const tc_pdr_spec* s, const tc_pdr_out* o, void* stream) {
  if (!h || !s || !o) return TC_EINVAL;
  if (s->nslab < 1 || s->ncell < 1 || s->nchunk < 1 || !s->n || !s->chi0 || !s->xi0 || !s->Z || !s->dx_cm)
    return TC_EINVAL;
  if (!(s->t_end_s >= 0.0) || !isfinite(s->t_end_s)) return TC_EINVAL;
  if (!all_finite_nonneg(s->n, s->nslab, true) || !all_finite_nonneg(s->dx_cm, s->nslab, true) ||
      !all_finite_nonneg(s->chi0, s->nslab, false) || !all_finite_nonneg(s->xi0, s->nslab, false) ||
      !all_finite_nonneg(s->Z, s->nslab, false))
    return TC_EINVAL;
  if (!start_state_ok(s->T_init, s->xH2_init, s->xHp_init)) return TC_EINVAL;
  const void* req[] = {o->T, o->x_h2, o->x_hp, o->x_e};
  for (const void* q : req)
    if (!q || !aligned8(q)) return TC_EINVAL;
  const void* opt[] = {o->x_co, o->chi_pe, o->f_shld_h2, o->N_c, o->N_trans};
  for (const void* q : opt)
    if (q && !aligned8(q)) return TC_EINVAL;
  if (h->p.mode == TC_MODE_MIXED_SEEDED || h->p.mode == TC_MODE_NEWTON_FP64_SEEDED) {
    if (!h->d_mlp) return TC_ENOMLP;
  }
  if ((double)s->nslab * (double)s->ncell > 9.0e15) return TC_EINVAL;
  const long long ncell = s->ncell * (long long)s->nslab;
  cudaStream_t st = (cudaStream_t)stream;
  const double* hp[5] = {s->n, s->chi0, s->xi0, s->Z, s->dx_cm};
  const size_t ns = (size_t)s->nslab;
  const size_t len[5] = {ns, ns, ns, ns, ns};
  double* dp[5];
  int rc0 = driver_setup(h, (size_t)ncell, hp, len, dp, st);
  if (rc0 != TC_OK) return rc0;

  tcg::PdrSlabs g;
  g.n = dp[0]; g.chi0 = dp[1]; g.xi0 = dp[2]; g.Z = dp[3]; g.dx = dp[4];
  g.nslab = s->nslab;
  g.ncell = s->ncell;
  g.T0 = s->T_init;
  g.xH20 = s->xH2_init;
  g.xHp0 = s->xHp_init;
  const size_t n = (size_t)ncell;
  tcg::DevFields f = driver_fields(h, n, o->T, o->x_h2, o->x_hp, o->x_e, o->x_co);
  tcg::PdrWork w;
  w.n = const_cast<double*>(f.n); w.chi_pe = const_cast<double*>(f.chi_pe); w.chi_lw = const_cast<double*>(f.chi_lw);
  w.fh2 = const_cast<double*>(f.fh2); w.xi = const_cast<double*>(f.xi); w.Zg = const_cast<double*>(f.Zg);
  w.Zd = const_cast<double*>(f.Zd); w.chi0 = const_cast<double*>(f.chi0);
  w.st = h->d_eqi; w.st_acc = h->d_eqi + n;
  const double dt = s->t_end_s / s->nchunk;
  for (int k = 0; k < s->nchunk; ++k) {
    if (tcg::launch_pdr_fields(g, w, o->T, o->x_h2, o->x_hp, k, false, nullptr, nullptr, nullptr, st) != cudaSuccess)
      return TC_ECUDA;
    h->launches += 1;
    f.hint = (k > 0) ? f.iters : nullptr;  // order each chunk by the previous chunk's iterations
    int rc = enqueue(h, false, f, ncell, dt, st);
    if (rc != TC_OK) return rc;
  }
  if (tcg::launch_pdr_fields(g, w, o->T, o->x_h2, o->x_hp, s->nchunk, true, o->chi_pe, o->f_shld_h2, o->N_c, st) !=
      cudaSuccess)
    return TC_ECUDA;
  h->launches += 1;
  if (o->status) {
    // the last launch's status OR-ed with the accumulated one
    if (cudaMemcpyAsync(o->status, w.st, n * sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return TC_ECUDA;
    if (tcg::launch_or_status(o->status, w.st_acc, ncell, st) != cudaSuccess) return TC_ECUDA;
    h->launches += 1;
  }
  if (o->N_trans) {
    if (tcg::launch_pdr_ntrans(g, o->x_h2, o->N_trans, st) != cudaSuccess) return TC_ECUDA;
    h->launches += 1;
  }
  return TC_OK;
}

