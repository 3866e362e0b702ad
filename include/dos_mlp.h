/*
 * dos_mlp.h -- the learned part of libdos: a small multilayer perceptron that
 * maps noisy low-order Chebyshev moments (mu_1..mu_{n_in} from a few start
 * vectors, as returned by dos_kpm_moments) to the density of states on a grid
 * (e.g. phi_hat at n_out Chebyshev nodes, as returned by dos_reconstruct).
 * The paper has no counterpart: it is an addition, scored against plain
 * Jackson-damped KPM (Appendix A) from the same few start vectors.
 *
 * Network:  h1 = relu(x W1^T + b1),  h2 = relu(h1 W2^T + b2),  y = h2 W3^T + b3
 * with W1 (n_hidden x n_in), W2 (n_hidden x n_hidden), W3 (n_out x n_hidden).
 * Loss: mean |y - target| (L1).  Optimiser: Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8) on FP32 master weights.  The matrix products run on tensor cores
 * with bfloat16 operands (weights, inputs, activations, back-propagated
 * gradients rounded to nearest-even) and FP32 accumulation; biases, losses,
 * bias gradients and the optimiser stay FP32.
 *
 * Parameters are exchanged as one flat FP32 array in the order
 * W1 (row-major), b1, W2, b2, W3, b3.  Arrays may be host or device memory.
 * All functions return DOS_* status codes (include/dos.h); messages go to the
 * owning context's dos_last_error().  Every wait inside the tensor-core
 * products is bounded: a wait that runs out skips that tile's stores and sets
 * a status flag of the network, which every call that synchronises (a host
 * output or loss, dos_mlp_get_params, dos_mlp_save) reads and clears,
 * returning DOS_ETIMEOUT; a call that stays asynchronous on a device stream
 * leaves the report to the next one that synchronises.  A dos_mlp is bound to
 * the context it was created from and must be destroyed before it.
 */
#ifndef DOS_MLP_H
#define DOS_MLP_H

#include <stdint.h>

#include "dos.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dos_mlp dos_mlp;

/* New network with He-uniform weights drawn from `seed` and zero biases.
 * 1 <= n_in, n_hidden, n_out <= 8192. */
int dos_mlp_create(dos_ctx *ctx, int n_in, int n_hidden, int n_out, uint64_t seed,
                   dos_mlp **out);
int dos_mlp_destroy(dos_mlp *mlp);

/* Number of parameters (the length of the flat parameter array). */
int dos_mlp_num_params(const dos_mlp *mlp, int64_t *count);

/* Replace all parameters; resets the Adam moments and step counter. */
int dos_mlp_set_params(dos_mlp *mlp, const float *params, void *stream);
/* Copy the FP32 master parameters out.  Synchronises `stream`. */
int dos_mlp_get_params(dos_mlp *mlp, float *params, void *stream);

/* y = network(x) for one training-sized batch: x is B x n_in, y is B x n_out
 * (row-major FP32), 1 <= B <= 65536; the activations stay in the network's
 * buffers (as dos_mlp_loss_grad leaves them).  Synchronises when y is host
 * memory. */
int dos_mlp_forward(dos_mlp *mlp, const float *x, int B, float *y, void *stream);

/* Inference: y = network(x) for any number of rows B >= 1.  Row r of x is the
 * n_in elements at x + r * ldx (ldx >= n_in; 0 means n_in) of type x_dtype
 * (DOS_F32, or DOS_F64 converted to FP32 on the device), so the network can
 * read mu_1..mu_{n_in} straight out of dos_kpm_moments_batched's output
 * (x = mu + 1, ldx = M + 1).  y: B x n_out row-major FP32.  Host or device
 * arrays.  Runs the forward kernels over consecutive slices of at most
 * `max_rows` rows (0: 8192), so the activation buffers stay bounded whatever B
 * is; each row's output is bitwise the same as dos_mlp_forward's for the same
 * FP32 input.  Synchronises when x or y is host memory. */
int dos_mlp_infer(dos_mlp *mlp, const void *x, int x_dtype, int64_t ldx, int64_t B, float *y,
                  int max_rows, void *stream);

/* Checkpoint: write the network to `path` in a byte-stable little-endian file:
 *   bytes 0-7   magic "DOSMLP\0\1" (format version 1)
 *   then int32 n_in, n_hidden, n_out, int32 0 (reserved), int64 Adam step count,
 *   int64 n_params, then n_params FP32 master parameters (the flat order above),
 *   n_params FP32 Adam first moments, n_params FP32 Adam second moments, and
 *   last a uint64 FNV-1a hash of every byte before it.
 * The same network state always gives the same bytes.  Synchronises `stream`.
 * Errors: DOS_EIO (cannot write), DOS_ECUDA, DOS_EINVAL. */
int dos_mlp_save(dos_mlp *mlp, const char *path, void *stream);

/* Create a network on `ctx` from a file written by dos_mlp_save: sizes,
 * parameters, Adam moments and step count restored, so inference and further
 * training continue bit for bit as from the saved network.  Errors: DOS_EIO
 * (cannot open or read, wrong magic or version, sizes that disagree with the
 * file length, or a hash mismatch), DOS_ENOMEM, DOS_ECUDA. */
int dos_mlp_load(dos_ctx *ctx, const char *path, dos_mlp **out, void *stream);

/* L1 loss of the batch and (if grads != NULL) its gradient with respect to
 * every parameter, flat FP32 in the parameter order.  No update.
 * loss: host pointer (may be NULL).  Synchronises `stream`. */
int dos_mlp_loss_grad(dos_mlp *mlp, const float *x, const float *target, int B, float *loss,
                      float *grads, void *stream);

/* One training step: forward, loss, backward and an Adam update with learning
 * rate lr > 0.  loss (host, may be NULL) receives the loss before the update
 * and makes the call synchronise; with loss == NULL the step stays
 * asynchronous. */
int dos_mlp_train_step(dos_mlp *mlp, const float *x, const float *target, int B, float lr,
                       float *loss, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DOS_MLP_H */
