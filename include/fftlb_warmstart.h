/* Learned warm start for the FFT-LB runs of arXiv:1011.3582 (Sec. 4:
 * phase separation of a van der Waals fluid from an unstable uniform
 * state).  A small convolutional network maps an early-time density and
 * temperature field, and the run temperature, to a later state of the same
 * run; the plain method (fftlb_step) continues from it.  The network is not
 * part of the paper; the method itself measures its error.
 *
 * Network (all spatial operations periodic, like the FFT-LB grid):
 *   input    X [3][H][W] float32:  X0 = s_rho (rho / rho_c - 1),
 *            X1 = s_T (T / T_run - 1),  X2 = T_run / T_c - 0.75
 *   layers   Z_l = b_l + W_l (*) A_{l-1}, with (*) the 3x3 periodic
 *            cross-correlation; A_l = max(Z_l, 0) for l = 1..3, A_0 = X;
 *            channels 3 -> 32 -> 32 -> 32 -> 2
 *   output   Y = Z_4 [2][H][W] float32, the predicted change of (X0, X1):
 *            rho' = rho_c (1 + (X0 + Y0) / s_rho),
 *            T'   = T_run (1 + (X1 + Y1) / s_T)
 *   loss     L = mean over 2 H W of (Y - (Xt - X[0:2]))^2 for a target Xt
 *            [2][H][W] (the later state encoded like X0, X1)
 *   training Adam (b1 = 0.9, b2 = 0.999, eps = 1e-8) on fp32 master
 *            parameters.
 * Arithmetic: the convolutions run on the tensor cores in bfloat16 with
 * fp32 accumulation.  Weights, A_0 and the stored activations A_1..A_3 are
 * rounded to bfloat16 (nearest even); Y is fp32.  Backward: the gradients
 * dL/dZ_l are rounded to bfloat16 before they multiply W_l or A_{l-1}; the
 * parameter gradients are accumulated in fp32.
 *
 * Parameter vector (fp32, FFTLB_CNN_NPARAMS floats): for l = 1..4 in order,
 * W_l [out][3][3][in] (row-major; tap (ky, kx) multiplies the value at
 * (y + ky - 1, x + kx - 1)) followed by b_l [out].
 *
 * Grids: 1 <= H, 64 <= W <= 4096 with W a multiple of 64.  Buffers of
 * fields are [c][H][W] row-major float32; `on_device` tells device pointers
 * (nonzero) from host pointers.  All work is queued on the stream given to
 * fftlb_cnn_create; calls that return host results synchronise it.  Every
 * call returns a status and never traps; fftlb_cnn_last_error describes
 * the last failure of that object (or of a failed create, with NULL). */
#ifndef FFTLB_WARMSTART_H
#define FFTLB_WARMSTART_H

#include "fftlb.h"

#ifdef __cplusplus
extern "C" {
#endif

#define FFTLB_CNN_NPARAMS (32 * 9 * 3 + 32 + 32 * 9 * 32 + 32 + 32 * 9 * 32 + 32 + 2 * 9 * 32 + 2)

typedef struct fftlb_cnn_s *fftlb_cnn_t;

/* Encoding constants: the EOS's critical density and temperature and the
 * input scales (s_rho = s_T = 50 are the defaults used by the tests). */
typedef struct {
    double rho_c, T_c, s_rho, s_T;
} fftlb_cnn_norm;

/* Allocates the activations, gradients and optimiser state for H x W
 * fields (about 400 bytes per site) and zero parameters.  FFTLB_ERR_ARG for
 * an unsupported grid, FFTLB_ERR_OOM if the device memory is short. */
fftlb_status fftlb_cnn_create(fftlb_cnn_t *c, int H, int W, void *cuda_stream);
fftlb_status fftlb_cnn_destroy(fftlb_cnn_t c);
const char *fftlb_cnn_last_error(fftlb_cnn_t c);

/* Host copies of the fp32 parameter vector.  set: reset_optimizer != 0
 * also zeroes the Adam moments and step count. */
fftlb_status fftlb_cnn_set_params(fftlb_cnn_t c, const float *params, int reset_optimizer);
fftlb_status fftlb_cnn_get_params(fftlb_cnn_t c, float *params);

/* Y = network(X).  X [3][H][W], Y [2][H][W]. */
fftlb_status fftlb_cnn_forward(fftlb_cnn_t c, const float *X, float *Y, int on_device);

/* Loss and its gradient with respect to the parameter vector (grad: host,
 * FFTLB_CNN_NPARAMS floats; either output may be NULL).  Xt [2][H][W]. */
fftlb_status fftlb_cnn_gradient(fftlb_cnn_t c, const float *X, const float *Xt, float *grad, double *loss,
                                int on_device);

/* One Adam step on the gradient of one sample; *loss (may be NULL)
 * receives the loss before the update. */
fftlb_status fftlb_cnn_train_step(fftlb_cnn_t c, const float *X, const float *Xt, float lr, double *loss,
                                  int on_device);

/* X (device, [3][H][W] float32) from the current rho, T of a handle of the
 * same grid, for the run temperature T_run (with X2 as above). */
fftlb_status fftlb_cnn_encode(fftlb_cnn_t c, fftlb_t h, double T_run, const fftlb_cnn_norm *norm, float *X_dev);

/* The warm start: encode the handle's current rho, T, run the network and
 * set the handle's state to f = f^eq(rho', u = 0, T') (the handle's step
 * count is kept). */
fftlb_status fftlb_cnn_warm_start(fftlb_cnn_t c, fftlb_t h, double T_run, const fftlb_cnn_norm *norm);

/* Kernel launches of the last forward / train step (for the bench's
 * launch count). */
long fftlb_cnn_launches(fftlb_cnn_t c);

#ifdef __cplusplus
}
#endif

#endif
