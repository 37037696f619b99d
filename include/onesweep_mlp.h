/*
 * onesweep_mlp.h - C ABI of the small cost model used for scheduling.
 *
 * Not part of the Onesweep method (the paper has no learned component). The
 * sort service can order waiting requests by predicted device time
 * (shortest first); the prediction comes from a one-hidden-layer perceptron
 *     pre = W1 x + b1,  h = max(pre, 0),  y = w2 . h + b2
 * trained on measured sort times. The network never sees keys, so sorted
 * outputs do not depend on it.
 *
 * Parameters are one float32 device array, laid out as
 *     W1 [hidden][features] (row-major), b1 [hidden], w2 [hidden], b2 [1]
 * (os_mlp_param_count() floats). Inputs x are float32 [n][features] row-major
 * (device), targets t and outputs y float32 [n] (device). features <= 32,
 * hidden <= 128. All calls enqueue on `stream` (a cudaStream_t, NULL = the
 * legacy default stream) and return an os_status value (include/onesweep.h):
 * OS_OK, OS_ERR_INVALID_ARG or OS_ERR_CUDA.
 */
#ifndef ONESWEEP_MLP_H
#define ONESWEEP_MLP_H

#include <stdint.h>

#include "onesweep.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Number of floats in the parameter array (0 for invalid sizes). */
OS_API int os_mlp_param_count(int features, int hidden);

/* y[i] = network(x[i]) for i < n. */
OS_API int os_mlp_forward(const float *params, int features, int hidden, const float *x, int n, float *y,
                          void *stream);

/*
 * Mean squared error L = (1/n) sum_i (y_i - t_i)^2 and its gradient with
 * respect to every parameter. grads (os_mlp_param_count floats) and *loss
 * (one float) are device memory; both are overwritten.
 */
OS_API int os_mlp_loss_grad(const float *params, int features, int hidden, const float *x, const float *t, int n,
                            float *grads, float *loss, void *stream);

/*
 * One Adam step (Kingma and Ba, 2015) on `count` parameters: m and v are the
 * first and second moment arrays (device, zero before step 1), step the
 * 1-based step number used for bias correction.
 */
OS_API int os_mlp_adam_step(float *params, const float *grads, float *m, float *v, int count, float lr, float beta1,
                            float beta2, float eps, int step, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ONESWEEP_MLP_H */
