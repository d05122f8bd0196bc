/*
 * tc_peak.h -- pipe-throughput microbenchmark kernels used to state the roofline of
 * the step kernels (not part of the step itself; the paper has no counterpart).
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
#ifdef __cplusplus
}
#endif
#endif
