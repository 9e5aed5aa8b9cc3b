/*
 * gsr_warm.h -- the learned warm start of libgsr: a small 1D convolutional
 * network over the attitude knot series that maps Jacobi-estimated attitude
 * parameters to an attitude guess, followed by per-star 5x5 least-squares
 * solves for the astrometric block. The paper has no warm start (its LSQR
 * starts from zero, Alg. 1); this is an addition of this library, and plain
 * LSQR from x0 = 0 remains available and is the reference.
 *
 * Network: 6 -> 64 -> 64 -> 64 -> 64 -> 64 -> 3 channels, kernel 5, zero
 * padding 2, ReLU after the first five layers; bf16 weights and activations,
 * fp32 accumulation on the tensor cores; fp32 master weights trained with
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error.
 * Parameters are exchanged as fp32 arrays: for each layer the weights
 * W[cout][cin][5] then the bias[cout] (gsr_net_num_params() values in all).
 * Sequence tensors are position-major fp32 [batch][len][channels] in device
 * memory. Conventions (status codes, streams) as in gsr.h.
 *
 * The convolution products (forward, backward-data, weight gradient) run as
 * tcgen05 MMAs into TMEM accumulators; each CTA waits at most 1 s for its MMAs. A convolution whose
 * wait runs out writes nothing, releases its TMEM and sets the net's fault
 * word: the next call on the net (forward, train_step, gradients, layer
 * calls), or gsr_lsqr_solve when its learned warm start ran the net, returns
 * GSR_ECUDA for it (gsr_net_gradients, which synchronises, also reports its
 * own). gsr_tc_wait_check (gsr.h) exercises that path.
 */
#ifndef GSR_WARM_H
#define GSR_WARM_H

#include <stdint.h>

#include "gsr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsr_net gsr_net;

/* number of network parameters (fp32 values) */
int64_t gsr_net_num_params(void);

/* gsr_net_create -- allocate a network on `device` (all parameters zero). */
gsr_status gsr_net_create(gsr_net **out, int32_t device);
gsr_status gsr_net_destroy(gsr_net *net);
const char *gsr_net_last_error(const gsr_net *net);

/* set / get the fp32 parameters (host arrays of gsr_net_num_params() values);
 * setting resets the Adam state. Synchronous. GSR_EINVAL on a count mismatch. */
gsr_status gsr_net_set_params(gsr_net *net, const float *params, int64_t count);
gsr_status gsr_net_get_params(gsr_net *net, float *params, int64_t count);

/* save / load the parameters to / from a file (a short header and the fp32 values) */
gsr_status gsr_net_save(gsr_net *net, const char *path);
gsr_status gsr_net_load(gsr_net *net, const char *path);

/*
 * gsr_net_forward -- out = net(in): in [batch][len][6], out [batch][len][3],
 * fp32 device arrays; each sequence is zero-padded at its own ends.
 */
gsr_status gsr_net_forward(gsr_net *net, const float *in, int64_t batch, int64_t len, float *out, void *stream);

/*
 * gsr_net_train_step -- one Adam step on the mean squared error between
 * net(in) and target ([batch][len][3] fp32, device); *loss (host, may be NULL)
 * receives the loss before the step. Synchronous when loss is not NULL.
 */
gsr_status gsr_net_train_step(gsr_net *net, const float *in, const float *target, int64_t batch, int64_t len,
                              float lr, double *loss, void *stream);

/*
 * gsr_net_gradients -- gradients of the mean squared error of one batch
 * (host array, same layout as the parameters) without updating the network.
 * Synchronous.
 */
gsr_status gsr_net_gradients(gsr_net *net, const float *in, const float *target, int64_t batch, int64_t len,
                             float *grads, int64_t count, double *loss, void *stream);

/*
 * gsr_net_layer_forward -- one layer of the network on caller data, for
 * checking the tensor-core convolution layer by layer: out = bias_l +
 * conv(W_l, in) before the ReLU and before any rounding of the output.
 * layer 0..5; in [batch][len][cin_l] fp32 device (rounded to bf16 as the
 * network rounds its layer inputs), out [batch][len][cout_l] fp32 device;
 * (cin_l, cout_l) = (6, 64), (64, 64) x 4, (64, 3). GSR_EINVAL on a bad layer.
 */
gsr_status gsr_net_layer_forward(gsr_net *net, int32_t layer, const float *in, int64_t batch, int64_t len, float *out,
                                 void *stream);

/*
 * gsr_net_layer_backward -- the gradients of one layer given dout =
 * dLoss/d(layer output before the ReLU), [batch][len][cout_l] fp32 device:
 * dout is rounded to bf16 for both products (as in training) and summed
 * unrounded for the bias gradient. din (NULL: skipped) [batch][len][cin_l]
 * fp32, not masked by the previous layer's ReLU; dW [cout_l][cin_l][5] and
 * db [cout_l] fp32 device, overwritten. The network's parameters and Adam
 * state are unchanged.
 */
gsr_status gsr_net_layer_backward(gsr_net *net, int32_t layer, const float *in, const float *dout, int64_t batch,
                                  int64_t len, float *din, float *dW, float *db, void *stream);

/*
 * gsr_net_apply_gradients -- one Adam step (as in gsr_net_train_step) with
 * caller-provided gradients: grads is a host fp32 array in the parameter
 * layout (count = gsr_net_num_params()), e.g. gradients summed over several
 * batches with gsr_net_gradients. Synchronous.
 */
gsr_status gsr_net_apply_gradients(gsr_net *net, const float *grads, int64_t count, float lr, void *stream);

/*
 * gsr_warm_features -- the network input of the loaded system: for every
 * attitude knot k (n_dfa rows) and axis a, the Jacobi estimate
 * (A^T b)_j / |A_:,j|^2 of column j = (a, k) divided by `scale` (the root mean
 * square of all 3*n_dfa Jacobi values), and log |A_:,j|^2 minus its mean over
 * the attitude columns: feats [n_dfa][6] fp32 (device). *scale (host) receives
 * the scale. Needs the rows and b. Synchronous.
 */
gsr_status gsr_warm_features(gsr_ctx *ctx, float *feats, double *scale, void *stream);

/*
 * gsr_warm_start -- the start vector x0 (n_cols binary64, device): attitude
 * part = scale * (features[:, 0:3] + net(features)) (net NULL: the Jacobi
 * estimate alone); instrumental and global parts = their Jacobi estimates
 * (A^T b)_j / |A_:,j|^2; astrometric part = per-star least squares (5x5) of
 * the rows' residual after all the other parts. Synchronous.
 */
gsr_status gsr_warm_start(gsr_ctx *ctx, gsr_net *net, double *x0, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GSR_WARM_H */
