/* sc_mlp.h -- the small multilayer perceptron that predicts, from a
 * subdomain's sparsity features, the run time and the error of every kernel
 * variant of the assembly (FP64, or split precision with 4..7 digits), so
 * that the variant can be chosen per subdomain without measuring it.  It is
 * trained on the timings and errors the autotuner records.  The paper has no
 * learned component; this is the learned part of the batched assembly.
 *
 * Network: x (n_in) -> ReLU(W1 x + b1) (n_hidden) -> ReLU(W2 h1 + b2)
 * (n_hidden) -> W3 h2 + b3 (n_out).  FP32.  Parameters are one contiguous
 * device array, in this order: W1 [n_hidden x n_in] row-major, b1, W2
 * [n_hidden x n_hidden], b2, W3 [n_out x n_hidden], b3.  Gradients and the
 * Adam moments use the same layout.
 *
 * Loss: masked mean squared error, L = sum_{b,o} mask (y - t)^2 / sum mask.
 *
 * All arrays are caller-owned device memory; batch rows are row-major
 * [batch x n]; calls are asynchronous on `stream` (a cudaStream_t).
 * Errors: 1 = invalid argument, 3 = CUDA launch error (codes of sc_status). */
#ifndef SC_MLP_H
#define SC_MLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n_in, n_hidden, n_out;
} sc_mlp_shape;

/* number of floats in the parameter array */
int64_t sc_mlp_param_count(const sc_mlp_shape *shape);

/* floats of device workspace needed for a batch (activations and their gradients) */
int64_t sc_mlp_workspace_floats(const sc_mlp_shape *shape, int32_t batch);

/* Y [batch x n_out] = network(X [batch x n_in]) */
int sc_mlp_forward(const sc_mlp_shape *shape, const float *params, const float *X, int32_t batch, float *Y,
                   float *ws, void *stream);

/* forward + backward: grads (same layout as params) = dL/dparams, and
 * loss[0] = L (device scalar).  T and mask are [batch x n_out]. */
int sc_mlp_loss_grad(const sc_mlp_shape *shape, const float *params, const float *X, const float *T,
                     const float *mask, int32_t batch, float *grads, float *loss, float *ws, void *stream);

/* one Adam step (Kingma & Ba 2015) over n parameters; step counts from 1 */
int sc_mlp_adam(int64_t n, float *params, const float *grads, float *m, float *v, float lr, float beta1,
                float beta2, float eps, int32_t step, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SC_MLP_H */
