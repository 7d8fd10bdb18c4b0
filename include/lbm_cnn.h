/*
 * lbm_cnn.h -- C ABI of the learned coarse-grid corrector.
 *
 * The paper has no learned component; this is an addition around its method.
 * A 5-layer convolutional network (3 x 3 kernels, channels 4 -> 32 -> 32 ->
 * 32 -> 32 -> 4, ReLU between layers, zero padding) maps the features
 * (log rho, u, v, log T) of a coarse MRT-FD run to a correction of the same
 * features: corrected = features + net(features). It is trained to match the
 * restriction (block means of rho, j, e) of a finer run of the same method.
 * Weights are stored in FP32 (Adam master copy). The first layer reads the
 * FP32 features and runs in FP32 (so that differences between neighbouring
 * nodes below one BF16 step are seen); the other layers use BF16 weights and
 * activations in tensor-core convolutions that accumulate in FP32, and the
 * correction is added to the FP32 features.
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

/* Loss (mean squared or absolute feature error against the target fields,
 * lbm_cnn_set_loss) and the
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

/* Training loss over the features of out = corrected, t = target, N values:
 * LBM_CNN_LOSS_MSE sum (out - t)^2 / N (default), LBM_CNN_LOSS_L1
 * sum |out - t| / N (the paper's error measure E of Sec. V.A is a relative
 * L1 norm). */
#define LBM_CNN_LOSS_MSE 0
#define LBM_CNN_LOSS_L1 1
int lbm_cnn_set_loss(lbm_cnn* n, int kind);

/* Output scale: the network predicts the correction of feature c (log rho,
 * u, v, log T) in units of scale[c] (corrected = features + scale * net),
 * host array of 4 values > 0; default 1. Setting it to the RMS correction
 * of the training data keeps the network's outputs of order one, so that
 * the rounding noise of its BF16 layers is a small fraction of the
 * corrections it has to produce. */
int lbm_cnn_set_output_scale(lbm_cnn* n, const double* scale);

/* rms[c] (host, 4 values) = root mean square over the image of the
 * difference target - coarse of feature c. Device fields [4][H][W].
 * Synchronises. */
int lbm_cnn_residual_rms(lbm_cnn* n, const double* coarse, const double* target, double* rms);

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
