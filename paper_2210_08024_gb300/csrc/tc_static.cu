// Host-buffer step that allocates nothing (declared in include/tc.h as
// tc_step_host_static).
//
// Who needs it: callers that hold their cell arrays in host memory but may not
// allocate device memory at all.  Examples are a code that runs inside another
// application's fixed device-memory budget, or a host code whose allocator is owned
// by someone else.  tc_step_host needs a handle (tc_create allocates its workspace)
// and device staging buffers that it allocates on first use.  This variant uses
// instead one statically sized scratch array in device global memory.  Every GPU that
// loads the library holds that array until the process exits.
//
// Scratch layout (doubles, TC_STATIC_MAX_CELLS = M):
//   [0, 9M)    inputs n, chi_pe, chi_lw, f_shld_h2, f_shld_c, F_lyc, xi_cr, Zg, Zd
//   [9M, 15M)  state and optional outputs T, x_h2, x_hp, x_e, x_cp, x_co
//   [15M, 16M) two int32 arrays, nsub and status
//   [16M]      work-queue cursor of the step kernel
// All calls share it: a call overwrites what the previous one left, and calls that
// overlap on the GPU (on different streams, or from different host threads) race.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/tc.h"
#include "tc_launch.h"

namespace tcg {
int occupancy_mode0_impl(int block);
int occupancy_mode1_impl(int block);
int occupancy_mode2_impl(int block);
}  // namespace tcg

namespace {

constexpr long long M = TC_STATIC_MAX_CELLS;
constexpr long long SCRATCH_DOUBLES = 16 * M + 32;

static __device__ __align__(256) double g_static_scratch[SCRATCH_DOUBLES];

// Device address of g_static_scratch, looked up once per device.  In host code the
// symbol's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with the device current.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_addr[MAX_DEVICES] = {nullptr};

int scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return TC_ENODEV;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return TC_ECUDA;
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return TC_OK;
}

tcg::DevParams to_dev(const tc_params& p) {
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

}  // namespace

extern "C" int tc_step_host_static(const tc_params* p, const tc_fields* f, double dt_s, void* stream) {
  if (!p || !f || f->ncell < 0) return TC_EINVAL;
  if (p->mode != TC_MODE_PAPER_FP64 && p->mode != TC_MODE_NEWTON_FP64 && p->mode != TC_MODE_MIXED)
    return TC_EINVAL;
  if (!(p->limiter > 0.0) || !(p->fd_rel_step > 0.0) || p->newton_max < 1 || p->max_substeps < 1)
    return TC_EINVAL;
  if (!(dt_s >= 0.0) || !isfinite(dt_s)) return TC_EINVAL;
  if (f->ncell > TC_STATIC_MAX_CELLS) return TC_EINVAL;  // beyond the static scratch
  if (f->ncell == 0) return TC_OK;
  if (!f->n || !f->chi_pe || !f->chi_lw || !f->f_shld_h2 || !f->xi_cr || !f->T || !f->x_h2 || !f->x_hp)
    return TC_EINVAL;
  if (!f->Zg && !(f->Zg_val >= 0.0)) return TC_EINVAL;
  if (!f->Zd && !(f->Zd_val >= 0.0)) return TC_EINVAL;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TC_ENODEV;
  double* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc != TC_OK) return rc;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TC_ECUDA;

  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)f->ncell;
  const double* hin[9] = {f->n, f->chi_pe, f->chi_lw, f->f_shld_h2, f->f_shld_c, f->F_lyc, f->xi_cr, f->Zg, f->Zd};
  double* din[9];
  for (int k = 0; k < 9; ++k) {
    din[k] = hin[k] ? base + (size_t)k * M : nullptr;
    if (hin[k] && cudaMemcpyAsync(din[k], hin[k], n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return TC_ECUDA;
  }
  double* hst[6] = {f->T, f->x_h2, f->x_hp, f->x_e, f->x_cp, f->x_co};
  double* dst[6];
  for (int k = 0; k < 6; ++k) {
    dst[k] = hst[k] ? base + (size_t)(9 + k) * M : nullptr;
    if (k < 3 && cudaMemcpyAsync(dst[k], hst[k], n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return TC_ECUDA;
  }
  int* ibase = (int*)(base + 15 * M);
  unsigned long long* cursor = (unsigned long long*)(base + 16 * M);
  // The cursor keeps the previous call's value: it must start at zero.
  if (cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st) != cudaSuccess) return TC_ECUDA;

  tcg::DevFields d;
  d.n = din[0]; d.chi_pe = din[1]; d.chi_lw = din[2]; d.fh2 = din[3]; d.fc = din[4]; d.Flyc = din[5];
  d.xi = din[6]; d.Zg = din[7]; d.Zd = din[8];
  d.T = dst[0]; d.xH2 = dst[1]; d.xHp = dst[2]; d.xe = dst[3]; d.xCp = dst[4]; d.xCO = dst[5];
  d.nsub = f->nsub ? ibase : nullptr;
  d.status = f->status ? ibase + M : nullptr;
  d.iters = nullptr;
  d.ncell = f->ncell;
  d.Zg_val = f->Zg_val;
  d.Zd_val = f->Zd_val;

  const int kmode = (p->mode == TC_MODE_PAPER_FP64) ? 0 : (p->mode == TC_MODE_MIXED) ? 2 : 1;
  int block = p->block > 0 ? p->block : 128;
  if (block > 128) block = 128;
  block = (block / 32) * 32;
  if (block < 32) block = 32;
  int per_sm = p->blocks_per_sm;
  if (per_sm <= 0)
    per_sm = (kmode == 0) ? tcg::occupancy_mode0_impl(block)
             : (kmode == 1) ? tcg::occupancy_mode1_impl(block) : tcg::occupancy_mode2_impl(block);
  long long grid = (long long)sms * per_sm;
  const long long need = (f->ncell + block - 1) / block;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  const tcg::DevParams dp = to_dev(*p);
  cudaError_t e;
  if (kmode == 0) e = tcg::launch_mode0(false, d, nullptr, dp, dt_s, cursor, f->ncell, (int)grid, block, st);
  else if (kmode == 1) e = tcg::launch_mode1(false, d, nullptr, dp, dt_s, cursor, f->ncell, (int)grid, block, st);
  else e = tcg::launch_mode2(false, d, nullptr, dp, dt_s, cursor, f->ncell, (int)grid, block, st);
  if (e != cudaSuccess) return TC_ECUDA;

  for (int k = 0; k < 6; ++k)
    if (hst[k] && cudaMemcpyAsync(hst[k], dst[k], n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return TC_ECUDA;
  if (f->nsub && cudaMemcpyAsync(f->nsub, d.nsub, n * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TC_ECUDA;
  if (f->status && cudaMemcpyAsync(f->status, d.status, n * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TC_ECUDA;
  return TC_OK;
}
