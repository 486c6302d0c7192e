/*
 * dtb_surrogate.h -- C ABI of the learned surrogate's MLP (part of libdtb.so).
 *
 * The surrogate maps a voxel's receptor hyper-parameters and summaries of the
 * previous assimilation window to the voxel's firing rate and BOLD in the
 * next window, so that the predict step of the hierarchical data assimilation
 * (section V.E) can run without the spiking simulation.  The paper has no
 * learned surrogate; the network is an extension of its assimilation loop.
 *
 * Network: x [B][n_in] -> (Linear -> GELU) x depth -> Linear -> y [B][n_out],
 * GELU(x) = 0.5 x (1 + erf(x / sqrt 2)).  Weights and activations are stored
 * in bfloat16, products accumulate in FP32 on the tensor cores, the pre-
 * activations, biases, gradients and Adam state are FP32.  Loss = mean squared
 * error over batch and outputs.  Parameters are one flat FP32 vector:
 * W_0 [n_in][width], b_0 [width], W_1 [width][width], b_1, ..., W_depth
 * [width][n_out], b_depth [n_out] (row-major).  Device memory is allocated
 * with cudaMalloc at creation; every call returns a dtb_status: DTB_EINVAL
 * for a NULL handle or array, sizes below 1, max_batch above 2^26 or a batch
 * B outside 1..max_batch; DTB_ENOMEM if creation cannot allocate; DTB_ECUDA
 * if a launch fails.  The compute calls wait for their work on the given
 * stream before returning.  Any sizes work: the GEMM tiles (64 x 64, k step
 * 16) read zeros beyond the edges.
 */
#ifndef DTB_SURROGATE_H
#define DTB_SURROGATE_H
#include <stdint.h>

#include "dtb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dtb_mlp dtb_mlp;

/* Creates the MLP with the given initial parameters (host FP32, layout above)
 * and buffers for batches of up to max_batch rows. */
dtb_status dtb_mlp_create(int32_t n_in, int32_t width, int32_t depth, int32_t n_out, int64_t max_batch,
                          const float* params, dtb_mlp** out);
dtb_status dtb_mlp_destroy(dtb_mlp* mlp);

/* Inference: d_x [B][n_in] FP32 device -> d_y [B][n_out] FP32 device. */
dtb_status dtb_mlp_forward(dtb_mlp* mlp, const float* d_x, float* d_y, int64_t B, void* stream);

/* Loss and gradients of the mean squared error to targets d_t [B][n_out]:
 * grads (host FP32, parameter layout) and *loss may each be NULL. */
dtb_status dtb_mlp_gradients(dtb_mlp* mlp, const float* d_x, const float* d_t, int64_t B, float* grads, float* loss,
                             void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr on the
 * gradients of this batch; *loss (may be NULL) is the batch loss before it. */
dtb_status dtb_mlp_train_step(dtb_mlp* mlp, const float* d_x, const float* d_t, int64_t B, float lr, float* loss,
                              void* stream);

/* Copies the FP32 master parameters to the host. */
dtb_status dtb_mlp_get_params(dtb_mlp* mlp, float* params);

#ifdef __cplusplus
}
#endif
#endif
