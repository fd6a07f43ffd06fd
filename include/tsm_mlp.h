/*
 * tsm_mlp.h -- the learned cost model's network: a 3-layer perceptron in
 * FP32 with hand-written CUDA forward, backward and Adam kernels.
 *
 * The paper finds kernel configurations by exhaustive search and names, as
 * future work, a performance model that would rank candidates from code
 * characteristics instead (Sec. 7).  This is that model's network.  It maps
 * a feature vector describing (shape, kernel variant, launch) to a predicted
 * cost; the tuner evaluates it for every candidate of an unseen shape and
 * keeps the argmin, with exhaustive search kept as its fallback and yardstick.
 *
 * Network:  h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = w3 . h2 + b3
 * with x in R^D (D <= TSM_MLP_MAX_IN), hidden width H (<= 64), scalar y.
 * Loss: mean squared error  L = (1/n) sum_i (y_i - t_i)^2.
 *
 * Parameter vector layout (host arrays of tsm_mlp_param_count() floats):
 *   W1 [H][D] row-major, b1 [H], W2 [H][H] row-major, b2 [H], w3 [H], b3 [1].
 * Gradients use the same layout.
 *
 * Ownership: the model owns its device buffers (parameters, gradients, Adam
 * moments, activations for up to max_batch samples); X (n x D row-major),
 * targets and outputs are caller-owned DEVICE float arrays.  Calls are
 * asynchronous on `stream` except the host<->device parameter copies, which
 * synchronize.  Every reduction over samples runs in sample order, so
 * training is bitwise reproducible.  Errors: INVALID_VALUE for null
 * pointers, n < 1 or n > max_batch, D or H out of range.
 */
#ifndef TSM_MLP_H
#define TSM_MLP_H

#include "tsm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define TSM_MLP_MAX_IN 32
#define TSM_MLP_MAX_HIDDEN 64

typedef struct tsm_mlp tsm_mlp;

/* Creates a model; weights drawn uniformly from +-1/sqrt(fan_in) with
 * SplitMix64 seeded by `seed`, biases zero, Adam moments zero. */
tsm_status tsm_mlp_create(int in_dim, int hidden, int max_batch, uint64_t seed, tsm_mlp **out);
void tsm_mlp_destroy(tsm_mlp *model);
int tsm_mlp_param_count(const tsm_mlp *model);

tsm_status tsm_mlp_set_params(tsm_mlp *model, const float *host_params);
tsm_status tsm_mlp_get_params(const tsm_mlp *model, float *host_params);
tsm_status tsm_mlp_get_grads(const tsm_mlp *model, float *host_grads);

/* y[i] = network(X[i]) for n samples. */
tsm_status tsm_mlp_forward(tsm_mlp *model, const float *X, int n, float *y, tsm_stream_t stream);

/* Forward + backward of the mean squared error over n samples: writes the
 * loss to *loss (device float) and the gradient into the model. */
tsm_status tsm_mlp_backward(tsm_mlp *model, const float *X, const float *target, int n,
                            float *loss, tsm_stream_t stream);

/* One Adam step (Kingma & Ba, 2015) on the current gradient, with bias
 * correction; step count kept by the model. */
tsm_status tsm_mlp_adam(tsm_mlp *model, float lr, float beta1, float beta2, float eps,
                        tsm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TSM_MLP_H */
