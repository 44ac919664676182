/*
 * surflbm_ws.h - learned warm start for the surfactant contact-line solver.
 *
 * The paper (Huang, Chai, Liu and Huang) has no counterpart of this part: it relaxes
 * every sessile drop from a cold start (a semicircle in uniform surfactant).  Here a
 * small convolutional encoder-decoder maps the parameters of a drop -- contact angle
 * theta0 of Eq. cos_angle, the solid-gas and solid-liquid adsorption strengths beta_sg,
 * beta_sl of Eq. boundary, the bulk surfactant load psi0 and the drop area -- to a
 * near-equilibrium (phi, psi) field, which is projected onto the conserved totals of the
 * cold start (sum psi of Eq. AC_psi's constraint, H = sum h_phi(phi) of Eq. conservation)
 * and used as the initial state; the lattice Boltzmann relaxation then finishes the job
 * and its step count measures the prediction.
 *
 * Network (fixed architecture, ny and nx divisible by 8):
 *   input 16 channels: the 5 normalised parameters and 11 fixed coordinate features
 *          (x, y, 1, x^2, y^2, xy, |x|, sin/cos(pi x / 2), sin/cos(pi y / 2); x, y scaled
 *          by ny / 2, x centred)
 *   level 0 (ny x nx):          conv 16->32, conv 32->32       (skip e0)
 *   level 1 (ny/2 x nx/2):      avgpool, conv 32->64, 64->64   (skip e1)
 *   level 2 (ny/4 x nx/4):      avgpool, conv 64->128, 128->128 (skip e2)
 *   level 3 (ny/8 x nx/8):      avgpool, conv 128->128, 128->128
 *   decoder: nearest upsample, concatenate the skip, two convs per level
 *            (256->128, 128->128; 192->64, 64->64; 96->32, 32->32)
 *   head   1 x 1 conv 32->2: phi and s = ln(psi / psi0)
 * Every 3 x 3 conv (zero padding, ReLU) runs on the tcgen05 tensor cores with BF16
 * weights and activations and FP32 accumulation; the master weights, Adam moments, the
 * head and the loss are FP32.  Loss: mean over cells of (phi - phi*)^2 + (s - s*)^2.
 *
 * Conventions as in surflbm.h.  "device" pointers are CUDA device memory owned by the
 * caller; "host" pointers are host memory read or written during the call only.  BF16
 * tensors are passed as uint16_t bit patterns.  Parameter rows (cond) are 5 floats:
 * theta0 [deg], beta_sg, beta_sl, psi0, area fraction (drop area / (nx ny)).
 */
#ifndef SURFLBM_WS_H
#define SURFLBM_WS_H

#include "surflbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- conv primitives
 * 3 x 3 convolution, stride 1, zero padding 1, NHWC: x [B][H][W][Cin] (BF16),
 * w [Cout][3][3][Cin] (BF16, tap (dy+1, dx+1) multiplies x[y+dy][x+dx]),
 * y [B][H][W][Cout].  Cin a multiple of 8, Cout a multiple of 16 in [16, 256]; all
 * device pointers 16-byte aligned.  Work is queued on stream (NULL = legacy default);
 * nothing is synchronised.  Kernel timeouts (a tensor-core wait that never ended)
 * raise a flag read by slbm_conv_error. */

/* y = act(conv(x, w) + bias); bias (FP32, Cout, may be NULL); relu 0/1. */
slbm_status slbm_conv3x3_forward(const uint16_t* x, const uint16_t* w, const float* bias, uint16_t* y, int B, int H,
                                 int W, int Cin, int Cout, int relu, void* stream);

/* wt [Cin][3][3][Cout] = w with taps mirrored and channels swapped (the weights of the
 * input-gradient convolution). */
slbm_status slbm_conv3x3_flip_weights(const uint16_t* w, uint16_t* wt, int Cin, int Cout, void* stream);

/* dx = (conv^T dy) * [mask > 0]: gradient w.r.t. x of sum(dy * conv(x, w)); wt from
 * slbm_conv3x3_flip_weights; mask [B][H][W][Cin] (may be NULL = no mask).  Cin a
 * multiple of 16 in [16, 256], Cout a multiple of 8. */
slbm_status slbm_conv3x3_input_grad(const uint16_t* dy, const uint16_t* wt, const uint16_t* mask, uint16_t* dx,
                                    int B, int H, int W, int Cin, int Cout, void* stream);

/* dw [Cout][3][3][Cin] (FP32) += gradient w.r.t. w of sum(dy * conv(x, w)).
 * Cout a multiple of 8 in [8, 128], Cin a multiple of 16 in [16, 256]. */
slbm_status slbm_conv3x3_weight_grad(const uint16_t* x, const uint16_t* dy, float* dw, int B, int H, int W, int Cin,
                                     int Cout, void* stream);

/* Synchronises the device; *flag = the primitives' timeout flag (0 = none); clears it. */
slbm_status slbm_conv_error(int* flag);

/* ---------------------------------------------------------------- network */
typedef struct slbm_ws slbm_ws;

/* Network for ny x nx fields and up to max_batch samples per call; weights drawn
 * (He-uniform, biases 0) from the counter-based generator with the given seed. */
slbm_status slbm_ws_create(int ny, int nx, int max_batch, unsigned long long seed, void* stream, slbm_ws** out);
long long slbm_ws_param_count(const slbm_ws* n);

/* FP32 master parameters, layer by layer: for each of the 14 convs w [Cout][3][3][Cin]
 * then b [Cout]; then the head w [2][32], b [2] (host, param_count floats). */
slbm_status slbm_ws_get_params(slbm_ws* n, float* host);
slbm_status slbm_ws_set_params(slbm_ws* n, const float* host);   /* also resets Adam */

/* out [B][2][ny][nx] (device FP32): phi and s = ln(psi / psi0) for the B parameter
 * rows cond (device, B x 5).  B <= max_batch. */
slbm_status slbm_ws_forward(slbm_ws* n, const float* cond, int B, float* out);

/* Loss and gradient of a minibatch: rows idx[0..B) (device ints; NULL = 0..B-1) of
 * cond (device, rows of 5) and targets (device, [rows][2][ny][nx] FP32: phi*, s*).
 * *loss (host) = the loss; grad (host, param_count floats, may be NULL) = its gradient. */
slbm_status slbm_ws_loss_grad(slbm_ws* n, const float* cond, const float* targets, const int* idx, int B,
                              double* loss, float* grad);

/* One Adam step on the gradient of the last slbm_ws_loss_grad call. */
slbm_status slbm_ws_adam(slbm_ws* n, float lr, float beta1, float beta2, float eps);

/* slbm_ws_loss_grad (without copying the gradient out) followed by slbm_ws_adam. */
slbm_status slbm_ws_train_step(slbm_ws* n, const float* cond, const float* targets, const int* idx, int B,
                               float lr, double* loss);

/* targets [2][ny][nx] (device) of instance idx of the batch at its current level:
 * phi and ln(psi / psi0) (the training target of that instance's equilibrium). */
slbm_status slbm_ws_batch_targets(slbm_ws* n, slbm_batch* b, int idx, double psi0, float* targets);

/* Warm start: every instance listed in which[0..count) (host ints) of the batch must be
 * ny x nx and freshly initialised with its cold-start fields (no step taken).  cond
 * (host, count x 5) are its parameters.  The prediction is projected onto the cold
 * start's sum psi and H (nonlinear constraint) or sum phi (linear) and becomes the
 * instance's initial state; accepted[k] (host, may be NULL) = 1, or 0 where the
 * projection failed and the cold start was kept. */
slbm_status slbm_ws_warm_start(slbm_ws* n, slbm_batch* b, const int* which, const float* cond, int count,
                               int* accepted);

size_t slbm_ws_device_bytes(const slbm_ws* n);
const char* slbm_ws_last_error(const slbm_ws* n);
void slbm_ws_destroy(slbm_ws* n);

#ifdef __cplusplus
}
#endif
#endif /* SURFLBM_WS_H */
