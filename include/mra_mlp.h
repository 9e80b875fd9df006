/*
 * mra_mlp.h -- C ABI of the learned surrogate of the MRA log-likelihood in
 * libmra.so: a multilayer perceptron 3 -> 64 -> 64 -> 1 with SiLU
 * activations that maps theta = (sigma2, beta, tau2) to a prediction of
 * loglik(theta) / n, trained on exact evaluations of mra_loglik.
 *
 * The surrogate is an addition to the method of the paper: the paper fits
 * theta by a derivative-free optimiser (BOBYQA, "likelihood" mode of
 * Sec. 2.2.5) that calls the exact log-likelihood at every step; here the
 * network proposes where the exact likelihood is evaluated next, and the
 * exact values decide on every proposal.
 *
 * Network (all sizes fixed):
 *   x_i  = 2 (log theta_i - log lo_i) / (log hi_i - log lo_i) - 1,  i = 0..2
 *   h1   = SiLU(W1 x + b1)          W1 [64][3],  b1 [64]
 *   h2   = SiLU(W2 h1 + b2)         W2 [64][64], b2 [64]
 *   yhat = w3 . h2 + b3             w3 [64],     b3 [1]
 *   prediction of loglik / n = t_off + t_scale * yhat
 * SiLU(z) = z / (1 + exp(-z)).  The parameters are held in FP32 ("master"
 * copy, updated by Adam) and in BF16; the forward and backward passes read
 * the BF16 copy and accumulate in FP32.
 *
 * Parameter vector (MRA_MLP_NPARAM floats, this order): W1 row-major,
 * b1, W2 row-major (W2[j][k] multiplies h1[k] into unit j), b2, w3, b3.
 *
 * Training loss over a set of B samples (theta_s, target_s):
 *   L = (1 / 2B) sum_s (yhat_s - (target_s - t_off) / t_scale)^2,
 * minimised by full-batch Adam (Kingma & Ba, 2015) with bias correction.
 *
 * Conventions: as in mra.h.  "Device" pointers are CUDA global memory on the
 * surrogate's device; calls on one surrogate must not overlap; nothing aborts,
 * traps or prints; mra_last_error(NULL) gives the reason of the last failure
 * on the calling thread.
 */
#ifndef MRA_MLP_H
#define MRA_MLP_H

#include <stddef.h>
#include <stdint.h>

#include "mra.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MRA_MLP_HIDDEN 64
#define MRA_MLP_NPARAM (3 * 64 + 64 + 64 * 64 + 64 + 64 + 1)

typedef struct mra_mlp mra_mlp;

typedef struct {
    double lo[3], hi[3];   /* theta box of the input scaling (all > 0, lo < hi) */
    double t_off, t_scale; /* target scaling: loglik/n = t_off + t_scale * yhat (t_scale > 0) */
} mra_mlp_scaling;

/* Create a surrogate on `device` with the given scaling and initial FP32
 * parameters (host, MRA_MLP_NPARAM floats; copied).  Adam moments start at 0.
 * EINVAL on a bad scaling or a null pointer; ECUDA/ENOMEM on device failure. */
mra_status mra_mlp_create(int device, const mra_mlp_scaling *scaling, const float *params, mra_mlp **out);

/* Replace the parameters (host, MRA_MLP_NPARAM floats) and reset Adam. */
mra_status mra_mlp_set_params(mra_mlp *m, const float *params);

/* Copy the FP32 master parameters to the host (MRA_MLP_NPARAM floats). */
mra_status mra_mlp_get_params(const mra_mlp *m, float *params);

/* Change the target scaling (the inputs' box is fixed at creation). */
mra_status mra_mlp_set_target_scaling(mra_mlp *m, double t_off, double t_scale);

/* Predictions of loglik/n at `batch` theta: theta_dev [batch][3] (FP64,
 * device), out_dev [batch] (FP64, device).  Asynchronous on `stream`
 * (a cudaStream_t, NULL for the legacy stream).  theta outside the box is
 * extrapolated; a non-positive component gives NaN. */
mra_status mra_mlp_predict(mra_mlp *m, const double *theta_dev, int batch, double *out_dev, void *stream);

/* Gradient of L at the current parameters over `batch` samples, without
 * updating anything: theta_dev [batch][3], target_dev [batch] (loglik/n,
 * FP64, device) -> grad_dev [MRA_MLP_NPARAM] (FP32, device) and *loss_dev
 * (FP32, device).  batch <= MRA_MLP_MAX_BATCH.  Asynchronous on `stream`. */
#define MRA_MLP_MAX_BATCH 65536
mra_status mra_mlp_grad(mra_mlp *m, const double *theta_dev, const double *target_dev, int batch, float *grad_dev,
                        float *loss_dev, void *stream);

/* `steps` full-batch Adam steps on the samples (theta_dev, target_dev) with
 * learning rate lr and the usual (beta1, beta2, eps) = (0.9, 0.999, 1e-8);
 * the step counter of the bias correction continues across calls until
 * mra_mlp_set_params.  loss_hist_dev (FP32, device, `steps` entries, may be
 * NULL) receives the loss at the parameters each step started from.  The
 * steps are replayed from a CUDA graph of the two kernels of one step.
 * Synchronous: returns when the last step has finished. */
mra_status mra_mlp_train(mra_mlp *m, const double *theta_dev, const double *target_dev, int batch, int steps,
                         float lr, float *loss_hist_dev);

void mra_mlp_free(mra_mlp *m);

#ifdef __cplusplus
}
#endif

#endif
