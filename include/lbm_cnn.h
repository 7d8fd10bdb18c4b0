/*
 * lbm_cnn.h -- C ABI of the learned coarse-grid corrector.
 *
 * The paper has no learned component; this is an addition around its method.
 * A 5-layer convolutional network (3 x 3 kernels, channels 4 -> 32 -> 32 ->
 * 32 -> 32 -> 4, ReLU between layers, zero padding) maps the features
 * (log rho, u, v, log T) of a coarse MRT-FD run to a correction of the same
 * features: corrected = features + net(features). It is trained to match the
 * restriction (block means of rho, j, e) of a finer run of the same method.
 * Weights are stored in FP32 (Adam master copy) and used in BF16 by the
 * tensor-core convolutions, which accumulate in FP32.
 *
 * Fields are 4 planes [4][H][W] (rho, u, v, T), FP64, row-major, x fastest.
 * Parameters are packed per layer as w[3][3][cin][cout] then b[cout], FP32,
 * layers in order (LBM_CNN_NPARAMS values in all).
 */
#ifndef LBM_CNN_H
#define LBM_CNN_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_CNN_LAYERS 5
#define LBM_CNN_NPARAMS 30084

typedef struct lbm_cnn lbm_cnn;

/* Network for H x W coarse grids (H, W >= 1, H * W <= 2^26); weights zero,
 * Adam state zero (lr 1e-3, betas 0.9 / 0.999, eps 1e-8). */
int lbm_cnn_create(int H, int W, void* cuda_stream, lbm_cnn** out);
int lbm_cnn_destroy(lbm_cnn* n); /* NULL-safe */

/* Parameters in the packed layout above; host or device FP32 arrays. */
int lbm_cnn_set_params(lbm_cnn* n, const float* params, int on_device);
int lbm_cnn_get_params(lbm_cnn* n, float* params, int on_device);
int lbm_cnn_set_adam(lbm_cnn* n, double lr, double beta1, double beta2, double eps);

/* Loss (mean squared feature error against the target fields) and the
 * gradient of every parameter (packed, FP32) for one coarse / target pair,
 * without updating. Fields: device pointers [4][H][W]. *loss and grads are
 * host outputs; synchronises. */
int lbm_cnn_loss_grad(lbm_cnn* n, const double* coarse, const double* target,
                      double* loss, float* grads);

/* One training step (forward, loss, backward, Adam update) on one pair of
 * device field arrays; *loss (host, may be NULL) receives the loss before the
 * update and synchronises when requested. */
int lbm_cnn_train_step(lbm_cnn* n, const double* coarse, const double* target,
                       double* loss);

/* Corrected fields [4][H][W] (device) from coarse fields (device). Falls back
 * to the plain coarse fields when the corrected total mass differs from the
 * coarse one by more than mass_tol (relative) or the output is not finite;
 * *used_fallback (host) tells which. Synchronises. */
int lbm_cnn_correct(lbm_cnn* n, const double* coarse, double* corrected,
                    double mass_tol, int* used_fallback);

/* Restriction of fine fields [4][Hf][Wf] (device) to [4][Hf/r][Wf/r] (device):
 * block means of rho, j_x, j_y, e over r x r blocks, then (rho, u, v, T).
 * Hf and Wf must be multiples of r. Asynchronous on cuda_stream. */
int lbm_restrict(const double* fine, int Hf, int Wf, int r, double* coarse,
                 void* cuda_stream);

const char* lbm_cnn_last_error(lbm_cnn* n);

#ifdef __cplusplus
}
#endif
#endif /* LBM_CNN_H */
