/*
 * tc.h -- C ABI of the GB300 thermochemistry source-step library.
 *
 * The library advances, cell by cell, the thermochemistry source step of Kim, Gong,
 * Kim & Ostriker (2023, arXiv:2210.08024), Sec. 6.1: with density and radiation frozen
 * over a time step dt, it subcycles the internal energy (through T_mu = T/mu) and the
 * non-equilibrium abundances x_H2 and x_H+ (Eqs. e:ODE1, e:ODE2), putting C+, CO, C, O,
 * O+ and the electrons in equilibrium after every substep (Secs. 3.2, 3.3) and using the
 * paper's rate coefficients (Sec. 3), heating (Sec. 4.1-4.4) and cooling (Sec. 4.3).
 *
 * Conventions
 *  - All functions return int: TC_OK (0) or a negative TC_E* code.  No C++ exception
 *    crosses this boundary.  tc_strerror() names a code.
 *  - Field arrays are caller-owned DEVICE pointers (SoA, FP64, length ncell, 8-byte
 *    aligned; 16-byte alignment lets the kernel use paired loads).  The library never
 *    frees or retains them after the call's kernels complete.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  All
 *    device work is stream-ordered; tc_step does not synchronise.
 *  - Per-cell numerical trouble (substep cap reached, Newton failure, non-finite state)
 *    does not fail the call: it is reported in the optional per-cell status array.
 *  - A handle is not thread-safe; use one handle per stream.
 *  - Only tc_step_host takes host pointers (it copies, runs and copies back).
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----- return codes */
#define TC_OK 0
#define TC_EINVAL (-1)    /* bad argument: NULL required pointer, ncell < 0, misalignment, bad mode */
#define TC_ECUDA (-2)     /* a CUDA runtime call failed; the sticky error is left to the caller */
#define TC_ENOMEM (-3)    /* device or host allocation failed */
#define TC_ENOMLP (-4)    /* seeded mode requested before tc_load_mlp */
#define TC_ENODEV (-5)    /* no sm_103 device visible */

/* ----- integration modes */
#define TC_MODE_PAPER_FP64 0   /* the paper's sequential update (Sec. 6.1), FP64 throughout */
#define TC_MODE_NEWTON_FP64 1  /* coupled backward Euler on (T_mu, x_H2, x_H+) by Newton, FP64 */
#define TC_MODE_MIXED 2        /* as TC_MODE_NEWTON_FP64: Newton iterations on FP32 source terms, FP64 residual,
                                  update and closure x_H; the substep length and a final polish of each
                                  root from double-float (df64) source terms */
#define TC_MODE_MIXED_SEEDED 3 /* as TC_MODE_MIXED, each Newton solve seeded by the MLP */
#define TC_MODE_NEWTON_FP64_SEEDED 4 /* as TC_MODE_NEWTON_FP64, MLP-seeded */

/* ----- physics switches (tc_params.flags) */
#define TC_CONST_KGR 1u  /* k_gr = 3e-17 Z'_d (the paper's test setting, Sec. 7) instead of Eq. e:H2form */
#define TC_NO_ROVIB 2u   /* H2 ro-vibrational cooling off (Sec. 7.1.2 comparison) */
#define TC_NO_CIE 4u     /* He + metal CIE cooling term of Eq. eq:cooling_fnct off */

/* ----- per-cell status bits.  Bits 1, 2 and 4 mark numerical trouble (tc_sync_status
 * counts cells with any of them); bits 8 and 16 are informational (mixed modes). */
#define TC_ST_MAX_SUBSTEPS 1
#define TC_ST_NEWTON 2       /* a Newton solve failed and the substep was halved */
#define TC_ST_NONFINITE 4
#define TC_ST_FALLBACK 8     /* a mixed solve did not converge; the FP64 Newton finished that substep */
#define TC_ST_POLISHED 16    /* a mixed solve stopped at the FP32 rounding floor before its df64 polish */
#define TC_ST_PREDICTOR 32   /* a Newton solve from the start state failed and was restarted from the
                                 block predictor (abundances by the 2x2 backward Euler, then T) */
#define TC_ST_SEEDED 64      /* seeded modes: a substep's solve started from the seed network converged */
#define TC_ST_SEED_FAIL 128  /* seeded modes: a seeded solve did not converge in 6 iterations and the
                                substep restarted from its start state (those iterations are counted) */
#define TC_ST_ERROR_MASK 7

typedef struct tc_params {
  double dvdr_kms_pc;          /* <|dv/dr|> in km/s/pc for CO trapping (Sec. 4.3.2); default 1 */
  double T_cmb;                /* radiation temperature floor of the dust (Sec. 4.3.6); default 2.73 K */
  double chi0;                 /* unattenuated FUV scale for optical dust heating; default 1 */
  double opt_over_fuv;         /* E_OPT,0 / E_FUV,0 (Sec. 4.3.6); default 1 */
  double tau_opt_over_tau_pe;  /* tau_OPT / tau_PE (Sec. 4.3.6); default 1/3 */
  double limiter;              /* factor of the substep rule (Sec. 6.1); default 0.1 */
  double fd_rel_step;          /* relative FD step for dH/dT_mu (mode 0); default 1e-3 */
  double newton_rtol;          /* Newton tolerance, FP64 modes; default 1e-12 */
  double T_floor;              /* temperature floor [K]; default 1 */
  int newton_max;              /* Newton iteration cap; default 50 */
  int max_substeps;            /* substep cap per cell; default 1e6 */
  int mode;                    /* TC_MODE_* */
  unsigned flags;              /* TC_CONST_KGR | TC_NO_ROVIB | TC_NO_CIE */
  double newton_rtol_mixed;    /* step tolerance of the FP32 Newton iterations of the mixed modes; default 1e-6
                                  (the df64 polish then brings each root to ~1e-9 relative) */
  int block;                   /* threads per block (0 = autotuned/default) */
  int blocks_per_sm;           /* resident blocks per SM for the persistent grid (0 = occupancy) */
  int order_cells;             /* 1 (default): hand cells to the persistent kernel in decreasing order of
                                  their predicted substep count, dt over the first substep length of
                                  Sec. 6.1 from the start-state sources (the library's scheduling, no
                                  counterpart in the paper; results are the same in any order, the
                                  longest cells then no longer finish last and warps hold cells of
                                  similar cost); needs 5 bytes of device workspace per cell, grown by
                                  cudaMalloc.  0: cells in index order. */
  int lanes_per_cell;          /* lanes that advance one cell together (the library's scheduling, no
                                  counterpart in the paper; results agree to rounding): 1, or 4 for the
                                  warp-cooperative kernels of modes TC_MODE_NEWTON_FP64 and TC_MODE_MIXED,
                                  whose four lanes evaluate the four points of each forward-difference
                                  Jacobian at once (tc_step and tc_step_host only; other modes and
                                  tc_step_batch use 1).  0 (default): for TC_MODE_NEWTON_FP64 and
                                  TC_MODE_MIXED 4 when the cells times 4 fit the cooperative kernel's
                                  resident lanes at once (launches too small to fill the GPU, whose
                                  time is the latency of the slowest cells), else 1, unless
                                  tc_autotune has recorded a choice for the launch's size class. */
} tc_params;

typedef struct tc_fields {
  /* inputs (device, length ncell) -- Table 1 of the paper */
  const double *n;          /* n_H [cm^-3] */
  const double *chi_pe;     /* chi_PE, Draine units (Eq. eq:chi_defn_PE) */
  const double *chi_lw;     /* chi_LW, dust-attenuated, no self-shielding (Eq. eq:chi_defn_LW) */
  const double *f_shld_h2;  /* f_shld,H2,eff; chi_H2 = chi_LW f (Eq. e:chi_H2) */
  const double *f_shld_c;   /* f_shld,C,eff; chi_C = chi_LW f (Sec. 5.1); may be NULL (= 1) */
  const double *F_lyc;      /* ionising photon flux c E_LyC/(h nu_LyC) [cm^-2 s^-1]; may be NULL (= 0) */
  const double *xi_cr;      /* primary CR ionisation rate per H [s^-1] */
  const double *Zg, *Zd;    /* per-cell Z'_g, Z'_d; may be NULL (then Zg_val, Zd_val) */
  /* state (device, in/out) */
  double *T, *x_h2, *x_hp;
  /* optional outputs (device, may be NULL) */
  double *x_e, *x_cp, *x_co;
  int *nsub, *status;
  long long ncell;
  double Zg_val, Zd_val;    /* scalars used when Zg / Zd are NULL */
  int *newton_iters;        /* optional out (device, may be NULL): Newton iterations summed over the
                               cell's substeps (modes 1-4; the mixed modes count FP32 iterations;
                               the seeded modes include abandoned seeded attempts) */
  const int *cost_hint;     /* optional in (device, may be NULL; tc_step and tc_step_batch only): a
                               per-cell cost estimate, larger = costlier, for example the newton_iters
                               output of the cell's previous step.  With tc_params.order_cells set,
                               cells are claimed in decreasing order of the hint instead of the
                               predicted substep count (in a simulation consecutive steps of a cell
                               cost about the same).  Results do not depend on it. */
} tc_fields;

typedef struct tc_handle tc_handle;

/* Fills *p with the defaults listed above for `mode`. */
int tc_params_default(tc_params *p, int mode);

/* Creates a handle on the current CUDA device: copies *p, allocates the small device
 * workspace (work-queue counter and status reduction).  *out is set only on success. */
int tc_create(const tc_params *p, tc_handle **out);

/* Enqueues one thermochemistry step of dt_s seconds for every cell of *f on `stream`.
 * Returns TC_EINVAL for NULL required pointers, ncell < 0, dt_s < 0 or a non-finite
 * dt_s; TC_ENOMLP for a seeded mode without weights; TC_ECUDA if the launch fails. */
int tc_step(tc_handle *h, const tc_fields *f, double dt_s, void *stream);

/* Enqueues one step for nbox independent boxes (each its own tc_fields, Z scalars and
 * size) as a single persistent-kernel launch over a device box table; on the first call
 * with a given box set the launch is captured into a CUDA graph that later identical
 * calls (same descriptors, dt_s, parameters and stream, compared in full) replay
 * without blocking.  A call with a different box set first waits on the host for the
 * cached graph's last launch to finish, since the box table's pinned host copy and
 * device copy are reused, then captures anew.  `boxes` is a host array of nbox
 * descriptors (1 <= nbox <= 64), read before the call returns.  Returns TC_EINVAL for a
 * bad count or descriptor, TC_ECUDA if capture or launch fails. */
int tc_step_batch(tc_handle *h, const tc_fields *boxes, int nbox, double dt_s, void *stream);

/* Start-state source terms of the substep rule (Sec. 6.1, with Eqs. e:ODE1, e:HH,
 * e:HII): for every cell of *f (device pointers as for tc_step; its state is only read)
 * the step's own start -- the C/O/e equilibrium at the input T, mu, T_mu -- and then
 * rate[3 i + 0] = C_H2, rate[3 i + 1] = C_H+ (the rates of change of x_H2 and x_H+,
 * s^-1) and rate[3 i + 2] = H / (K T_mu) (that of ln T_mu, s^-1), all FP64, and
 * dts[i] = the length in seconds of the first substep of a step of dt_s.  rate (3 ncell
 * doubles) and dts (ncell doubles) are device arrays; either may be NULL.  Enqueued on
 * `stream`.  These are the explicit-Euler rates that the seed network takes as inputs
 * (tc_mlp.h).  Returns TC_EINVAL for bad fields or dt_s, TC_ECUDA if the launch fails. */
int tc_rates(tc_handle *h, const tc_fields *f, double dt_s, double *rate, double *dts, void *stream);

/* Launch shape chosen by tc_autotune (the library's scheduling; the paper has no
 * counterpart). */
typedef struct tc_tune_choice {
  int block;           /* threads per block */
  int blocks_per_sm;   /* resident blocks per SM of the persistent grid (0 = occupancy limit) */
  int lanes_per_cell;  /* 1, or 4 for the warp-cooperative kernels */
  float ms;            /* time of one step of *f in that shape */
} tc_tune_choice;

/* Autotuner of the step launch.  Times one step of the cells of *f (device pointers, as
 * for tc_step) in every candidate shape -- 32, 64 or 128 threads per block, the occupancy
 * limit or 4 resident blocks per SM, and for modes TC_MODE_NEWTON_FP64 and TC_MODE_MIXED
 * one or four lanes per cell (four only when the cooperative kernel holds the cells in
 * at most 8 waves of its resident lanes) -- with CUDA events on `stream`, each candidate
 * once, or three times (fastest kept) when one step takes under 20 ms, and records the fastest
 * for the size class floor(log2(ncell)) in the handle: later tc_step and tc_step_host
 * calls of that size class whose tc_params leave block, blocks_per_sm and
 * lanes_per_cell at 0 use it.  The candidates advance a scratch copy of T, x_h2 and
 * x_hp (allocated here by cudaMalloc and freed before returning): *f is not modified.
 * Synchronises `stream`; not for use while `stream` is being captured.  Writes the
 * choice to *best.  Returns TC_EINVAL for bad fields, ncell < 1 or a bad dt_s,
 * TC_ENOMLP for a seeded mode without weights, TC_ENOMEM, or TC_ECUDA. */
int tc_autotune(tc_handle *h, const tc_fields *f, double dt_s, void *stream, tc_tune_choice *best);

/* Like tc_step but every pointer in *f is a HOST pointer: the call copies inputs to the
 * device, runs the step, copies T, x_h2, x_hp (and the optional outputs) back and
 * synchronises `stream` before returning. */
int tc_step_host(tc_handle *h, const tc_fields *f, double dt_s, void *stream);

/* Largest ncell that tc_step_host_static accepts. */
#define TC_STATIC_MAX_CELLS 65536

/* tc_step_host_static -- the paper has no counterpart: this is a service of the library.
 * It is tc_step_host for callers that may not allocate device memory: for instance a code
 * running inside another application's fixed device-memory budget, or one whose device
 * allocator belongs to someone else.  It needs no handle and calls no cudaMalloc or
 * cudaFree.  Its device staging (inputs, state, outputs) and the work-queue cursor of the
 * step kernel live in one file-scope device array sized for TC_STATIC_MAX_CELLS cells
 * (~8.4 MB).  Every GPU that loads the library holds that array until the process exits.
 *  - p: parameters as for tc_create (modes TC_MODE_PAPER_FP64, TC_MODE_NEWTON_FP64 and
 *    TC_MODE_MIXED; seeded modes are rejected).  f: HOST pointers as for tc_step_host.
 *  - Copies the inputs in, runs one step of dt_s seconds on `stream`, copies T, x_h2,
 *    x_hp and the optional outputs back, and synchronises `stream` before returning.
 *  - Returns TC_EINVAL if ncell > TC_STATIC_MAX_CELLS, for NULL required pointers, a bad
 *    mode or a negative or non-finite dt_s; TC_ECUDA if a CUDA call fails.
 *  - The first call on a device looks up the array's device address (once per device,
 *    with that device current).  Make that first call before any stream capture.
 *  - All calls share the array, and each call overwrites what the last one left.  Calls
 *    that overlap on the GPU (other streams or host threads) race: serialise them. */
int tc_step_host_static(const tc_params *p, const tc_fields *f, double dt_s, void *stream);

/* Loads the seed network's weights (the blob written by tc_mlp_export, include/tc_mlp.h,
 * exactly tc_mlp_blob_bytes() bytes) into the handle; TC_EINVAL for a blob of another
 * size or layout version.  Required before a step in a seeded mode. */
int tc_load_mlp(tc_handle *h, const void *blob, size_t bytes);

/* The seed network as the seeded step kernels evaluate it: warp-level BF16 tensor-core
 * inference (mma.sync m16n8k16, FP32 accumulation; inputs and hidden activations rounded
 * to BF16) of the network loaded by tc_load_mlp, on B rows of raw features X[B][13]
 * (device, float32, in the order of tc_mlp.h), writing out[B][3] (device, float32) on
 * `stream`.  The paper has no counterpart; this is the library's check of its
 * inference.  Returns TC_EINVAL for B < 0 or NULL arrays, TC_ENOMLP without weights,
 * TC_ECUDA if the launch fails. */
int tc_seed_predict(tc_handle *h, const float *X, int B, float *out, void *stream);

/* Counts cells whose status has any TC_ST_ERROR_MASK bit in the last step's status array
 * on `stream` and synchronises it; *nbad receives the count. */
int tc_sync_status(tc_handle *h, const int *status, long long ncell, void *stream, long long *nbad);

/* Number of device kernel launches the handle has issued (for accounting). */
long long tc_launch_count(const tc_handle *h);

const char *tc_strerror(int code);

void tc_destroy(tc_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* TC_H */
