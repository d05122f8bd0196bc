/*
 * tc_mlp.h -- training and export of the seed network of the implicit solve.
 *
 * The seeded modes (TC_MODE_MIXED_SEEDED, TC_MODE_NEWTON_FP64_SEEDED) start every
 * substep's Newton iteration from the prediction of a small network instead of from the
 * substep's start state.  The solve still runs to its own convergence criterion, so the
 * result is the same root; the network only shortens the path to it.  The paper has no
 * learned component: this is the build's acceleration of its coupled implicit scheme
 * (Sec. 6.1).
 *
 * Network: 13 features -> 64 -> 64 -> 64 (SiLU) -> 3 outputs.
 *   features: log10 n, log10 T, x_H2, x_H+, log10 chi_FUV, log10 f_shld,H2,
 *             log10(F_LyC + 1), log10 xi_cr, log10 dt, log10 Z'_d, and the explicit-Euler
 *             changes over the step g = dt (C_H2 / 0.5, C_H+, H / (K T_mu ln 10)) from the
 *             start-state source terms (tc_rates in tc.h)   (raw; normalised inside with
 *             the mean and standard deviation given to tc_mlp_set_norm)
 *   outputs:  changes over one backward-Euler step of length dt (the implicit solve's
 *             root) minus g: (x_H2' - x_H2)/0.5 - g0, x_H+' - x_H+ - g1,
 *             log10 T' - log10 T - g2
 * Parameters: one FP32 master vector of tc_mlp_n_params() floats, in the order
 *   W1[64][13], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[3][64], b4[3].
 * The forward and backward passes use the weights rounded to BF16 and accumulate in
 * FP32.  Training is Adam on the FP32 masters.
 *
 * Pointers named X, Y, grad, loss, out are DEVICE pointers (row-major, B rows); theta,
 * mean, stdev and blob are host pointers.  All calls return TC_OK or a negative TC_E*
 * code from tc.h.  A handle is not thread-safe.
 */
#ifndef TC_MLP_H
#define TC_MLP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_mlp tc_mlp;

/* Number of FP32 parameters (9411). */
int tc_mlp_n_params(void);

/* Creates a network on the current device: uniform initialisation with bound
 * sqrt(6/fan_in) from a splitmix64 stream seeded by `seed`, zero biases, zero Adam
 * state, identity normalisation. */
int tc_mlp_create(unsigned long long seed, tc_mlp **out);
void tc_mlp_destroy(tc_mlp *h);

/* Feature normalisation (f - mean) / stdev; stdev must be > 0. */
int tc_mlp_set_norm(tc_mlp *h, const float *mean, const float *stdev);

/* Copies the FP32 masters in or out (host arrays of tc_mlp_n_params() floats). */
int tc_mlp_set_params(tc_mlp *h, const float *theta);
int tc_mlp_get_params(const tc_mlp *h, float *theta);

/* out[B][3] = network(X[B][13]) on `stream`. */
int tc_mlp_predict(tc_mlp *h, const float *X, int B, float *out, void *stream);

/* Gradient of the weighted mean-squared error sum_m w_m (o_m - y_m)^2 / B with respect
 * to the parameters (written to grad, tc_mlp_n_params() floats) and the loss (one
 * float), both on the device.  w3 is a host array of 3 weights or NULL (all ones).
 * grad or loss may be NULL. */
int tc_mlp_grad(tc_mlp *h, const float *X, const float *Y, int B, const float *w3, float *grad, float *loss,
                void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on the batch; the
 * batch loss before the step goes to *loss (device) when loss is not NULL. */
int tc_mlp_train_step(tc_mlp *h, const float *X, const float *Y, int B, const float *w3, float lr, float *loss,
                      void *stream);

/* Size of the weight blob that tc_load_mlp (tc.h) accepts. */
size_t tc_mlp_blob_bytes(void);

/* Writes the blob (BF16 weights in the step kernel's layout, FP32 biases and the
 * normalisation) into a host buffer of at least tc_mlp_blob_bytes() bytes. */
int tc_mlp_export(const tc_mlp *h, void *blob, size_t cap);

#ifdef __cplusplus
}
#endif
#endif /* TC_MLP_H */
