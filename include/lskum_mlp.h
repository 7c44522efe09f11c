/*
 * lskum_mlp.h -- learned warm start for the q-LSKUM solver of lskum.h.
 *
 * No counterpart in the paper (Verma, Mamidi and Nemili 2024 start every
 * solve from the free stream; Sec. 5).  This extension predicts an initial
 * flow field with a small network trained on converged solutions that the
 * solver itself produced; the solver's own residual decides, per case,
 * whether the prediction or the free stream is used.
 *
 * Network (all values per point):
 *   z = (zeta_x, zeta_y, delta): the position relative to mid-chord
 *       compactified into the unit disc, (x - 0.5, y) / (1 + r) with
 *       r = |(x - 0.5, y)|, and the wall distance d as d / (1 + d), where d
 *       is the distance to the case's wall polygon (wall points in caller
 *       order, closed);
 *   inputs = [sin 2 pi B z, cos 2 pi B z, M, AoA / 10 deg] (34 values; B is
 *       a fixed 16x3 matrix drawn N(0, 1) at create);
 *   34 -> 128 -> 128 -> 128 -> 128 -> 4, GELU (erf form) after each hidden
 *       layer; outputs o -> rho = exp(o0), u = u_inf + o1, v = v_inf + o2,
 *       p = p_inf exp(o3).
 * Arithmetic: every matrix product runs on the tensor cores (tcgen05, BF16
 * operands, FP32 accumulation in tensor memory): inputs, weights, hidden
 * activations and back-propagated gradients are rounded to BF16 (nearest
 * even) where they enter a product; biases, GELU, the loss, the optimiser
 * (Adam, FP32 master weights) and the output map are FP32.
 *
 * Parameters are exchanged as one FP32 vector: for each layer l = 0..4 its
 * weights W_l [out][in] (row-major, in = 34 for l = 0) then its biases
 * b_l [out]; lskum_mlp_n_params() values in total.
 *
 * All pointers are host pointers unless a name ends in _dev.  Every call
 * returns a status; a failure leaves the object valid.  An object is used by
 * one host thread at a time.
 */
#ifndef LSKUM_MLP_H
#define LSKUM_MLP_H

#include "lskum.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lskum_mlp lskum_mlp; /* opaque, owned by the library */

/* Number of FP32 values in the parameter vector (54,532). */
int32_t lskum_mlp_n_params(void);

/* Create a network: weights and biases uniform in +-1/sqrt(fan_in) and the
 * Fourier matrix B from `seed`; buffers for training batches of up to
 * max_batch samples (rounded up to a multiple of 512; >= 512).
 * cuda_stream: a stream of the current device or NULL.  Errors: LSKUM_ERR_ARG,
 * LSKUM_ERR_OOM, LSKUM_ERR_CUDA. */
lskum_status lskum_mlp_create(uint64_t seed, int32_t max_batch, void *cuda_stream, lskum_mlp **out);

/* Copy the parameters (n_params floats) and B (48 floats, row-major 16x3;
 * may be NULL) out of / into the network.  set_params also resets Adam. */
lskum_status lskum_mlp_get_params(lskum_mlp *m, float *params, float *fourier);
lskum_status lskum_mlp_set_params(lskum_mlp *m, const float *params, const float *fourier);

/* Network inputs of n points: in5 [n][5] = (x, y, wall distance, M, AoA deg)
 * -> X [n][34] (the BF16-rounded values the first product reads). */
lskum_status lskum_mlp_features(lskum_mlp *m, const float *in5, int32_t n, float *X);

/* Forward pass from given inputs X [n][34] (rounded to BF16 on entry), any n
 * >= 0: out [n][4] = the outputs o. */
lskum_status lskum_mlp_forward(lskum_mlp *m, const float *X, int32_t n, float *out);

/* Mean squared error of the outputs for inputs X [n][34] against targets
 * T [n][4] (1 <= n <= max_batch) and its gradient with respect to the
 * parameters (grads: n_params floats, same layout). */
lskum_status lskum_mlp_loss_grads(lskum_mlp *m, const float *X, const float *T, int32_t n, float *loss,
                                  float *grads);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the
 * given gradient vector (n_params floats) and learning rate. */
lskum_status lskum_mlp_adam(lskum_mlp *m, const float *grads, float lr);

/* Measure: mean device time (CUDA events on the network's stream) of the
 * forward pass over n points (in chunks of max_batch), reps repetitions, on
 * whatever inputs the buffers hold (the products' cost does not depend on
 * the values).  The network's parameters are unchanged. */
lskum_status lskum_mlp_time_forward(lskum_mlp *m, int32_t n, int32_t reps, double *ms);

/* Append training samples from the context's current state: per case,
 * per_case points drawn without replacement (seeded; all points of a case if
 * it has fewer) among its wall and interior points, skipping cases whose
 * status is not LSKUM_OK.  Inputs (x, y, wall distance, M, AoA) and targets
 * (log rho, u - u_inf, v - v_inf, log(p / p_inf)) stay on the device. */
lskum_status lskum_mlp_add_samples(lskum_mlp *m, lskum_ctx *ctx, int32_t per_case, uint64_t seed);

/* Number of stored samples. */
lskum_status lskum_mlp_n_samples(lskum_mlp *m, int32_t *n);

/* Train for `epochs` passes over the stored samples in shuffled batches of
 * `batch` (<= max_batch) samples (the last batch of an epoch may be smaller),
 * Adam with learning rate lr; epoch_loss[epochs] (may be NULL) receives each
 * epoch's mean batch loss. */
lskum_status lskum_mlp_train(lskum_mlp *m, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                             float *epoch_loss);

/* Warm start: predict the state of every case of ctx (wall and interior
 * points; outer points keep the free stream), then let the residual judge:
 * for each case whose first residual norm from the prediction is not below
 * the free stream's, the free stream is used instead.  The history is cleared
 * as by lskum_set_state.  warm[n_cases] (may be NULL) receives 1 where the
 * prediction was kept.  Errors as lskum_set_state. */
lskum_status lskum_mlp_predict(lskum_mlp *m, lskum_ctx *ctx, int32_t *warm);

/* Distance of every point of ctx to its case's wall polygon (f64[N], caller
 * order), as the network sees it (computed in FP32 on the device). */
lskum_status lskum_get_wall_distance(lskum_ctx *ctx, double *d);

/* Number of first-order start-up iterations (lskum_opts.first_order_iters)
 * for the runs that follow; iterations are counted from the last new state. */
lskum_status lskum_set_start_iters(lskum_ctx *ctx, int32_t first_order_iters);

/* Failure-path test of the tensor-core waits (no counterpart in the paper).
 * Every wait of the network's kernels for its tensor-core products is
 * bounded: past wait_limit_s (1 s by default) the kernel gives up, frees its
 * tensor memory and returns, and the call reports LSKUM_ERR_TIMEOUT with the
 * object still usable.  skip_products = 1 makes the product kernels issue
 * neither the products nor the commit that would complete the wait, so the
 * wait runs out with nothing in flight; 0 restores normal operation.
 *   skip_products  0 or 1
 *   wait_limit_s   1e-4 .. 10 seconds, applied to every later call
 * Errors: LSKUM_ERR_ARG. */
lskum_status lskum_mlp_set_wait_test(lskum_mlp *m, int32_t skip_products, double wait_limit_s);

/* Message of the last failure of m; never NULL. */
const char *lskum_mlp_last_error(const lskum_mlp *m);

/* Free everything; NULL is allowed. */
void lskum_mlp_destroy(lskum_mlp *m);

#ifdef __cplusplus
}
#endif

#endif /* LSKUM_MLP_H */
