/*
 * tc_peak.h -- pipe-throughput microbenchmark kernels used to state the roofline of
 * the step kernels, and the device check of the df64 arithmetic (not part of the step
 * itself; the paper has no counterpart).
 *
 * tc_peak_launch enqueues `kind` on `stream`: grid x block threads each run `chains`
 * independent dependency chains of `iters` operations.  The caller times it (CUDA
 * events on the same stream).  Operations per launch = grid * block * chains * iters.
 *   kind 0: FP64 fused multiply-add      kind 1: FP32 fused multiply-add
 *   kind 2: FP64 exp()                   kind 3: FP64 log()
 *   kind 4: FP64 sqrt()                  kind 5: FP64 division
 *   kind 6: FP64 pow(x, y)               kind 7: FP32 expf()
 *   kind 8: FP32 __expf(), the approximate exponential of the fast-math mixed kernels:
 *           one MUFU ex2 per operation, so its rate is the MUFU pipe's
 *   kind 9: df64 (double-float) multiply then add, v = v a + b: the mixed kernels'
 *           high-precision arithmetic on the FP32 pipes (one operation = one multiply
 *           and one add)
 *   kind 10: df64 exp()
 * `sink` is a device buffer of grid * block doubles that receives the chain results
 * (written so the compiler cannot drop the work).  Returns TC_OK, TC_EINVAL or TC_ECUDA.
 */
#ifndef TC_PEAK_H
#define TC_PEAK_H
#ifdef __cplusplus
extern "C" {
#endif
int tc_peak_launch(int kind, int grid, int block, int iters, double *sink, void *stream);
int tc_peak_chains(void);

/*
 * tc_df64_eval -- element-wise df64 (double-float: a value is the unevaluated sum of two
 * FP32 numbers, ~44-48 significant bits) arithmetic on the device, compiled like the
 * mixed-precision step kernels that use it (fast FP32 intrinsics, flush-to-zero), for
 * accuracy tests against FP64.  Each input is converted from FP64 to df64, the result
 * back to FP64:
 *   op 0: a + b   op 1: a * b   op 2: a / b   op 3: sqrt(a)   op 4: exp(a)   op 5: log(a)
 * a, b (b only for ops 0-2; may be NULL otherwise) and out are device arrays of n
 * doubles; enqueued on `stream`.  Returns TC_OK, TC_EINVAL or TC_ECUDA.
 */
int tc_df64_eval(int op, const double *a, const double *b, double *out, long long n, void *stream);

/*
 * tc_df64_source_check -- the heating/cooling and chemistry source terms of every cell of
 * f at its stored state (T, x_H2, x_H+; C/O/e equilibrium and dust temperature solved),
 * evaluated in df64 as the mixed kernels' polish does and in FP64, on the device.
 * err (device, 5 * ncell doubles, SoA) receives per cell:
 *   [0] |H_df - H| / (n G + n^2 |L|)       (H = n G - n^2 L, Eq. e:ODE1's source)
 *   [1] |C_H2,df - C_H2| / (formation + destruction)
 *   [2] |C_H+,df - C_H+| / (ionisation + recombination)
 *   [3] relative error of the dust temperature,  [4] of x_e.
 * p supplies the physics parameters (mode ignored); f's state is read only.  Enqueued
 * on `stream`.  Returns TC_OK, TC_EINVAL (NULL or misaligned pointers) or TC_ECUDA.
 */
struct tc_params;
struct tc_fields;
int tc_df64_source_check(const struct tc_params *p, const struct tc_fields *f, double *err, void *stream);
#ifdef __cplusplus
}
#endif
#endif
