/*
 * resnet.h -- C ABI of the transmit-side ResNet generator z = f_theta(y0)
 * (Eq. 17, Section III-A; the architecture of Section IV: 5 residual blocks of
 * hidden width 128, tanh in the hidden and residual layers, sigmoid output).
 *
 *   h_0 = tanh(W_in y0 + b_in)
 *   r_k = tanh(W1_k h_{k-1} + b1_k),  h_k = tanh(h_{k-1} + W2_k r_k + b2_k),  k = 1..5
 *   u   = W_out h_5 + b_out,          z = sigmoid(u)
 *
 * P = N M phases (y0 = vec(Y0) of Eq. 16, values in [0, 1]).  u is the
 * pre-sigmoid output: it takes the place of the direct logits of sqngd.h,
 * so the rest of the transmit chain (Eqs. 23, 24, 43) is unchanged.
 *
 * Parameters: one float vector of rn_param_count(P) entries in the order
 * W_in [128][P], b_in [128], then for k = 1..5: W1_k [128][128], b1_k [128],
 * W2_k [128][128], b2_k [128], then W_out [P][128], b_out [P]; matrices
 * row-major.  Adam state lives in the handle (beta1 0.9, beta2 0.999,
 * eps 1e-8 for rn_train_step; the step of sqngd_step uses the context's).
 *
 * Device pointers are CUDA device memory on the current device; host
 * pointers are ordinary memory.  Calls are asynchronous on the handle's
 * stream unless noted.  Every function returns an af_status (sqngd.h).
 */
#ifndef PAPER_2604_25728_RESNET_H
#define PAPER_2604_25728_RESNET_H

#include <stdint.h>

#include "sqngd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rn_net rn_net;

/* Number of parameters for P phases, or -1 if P < 1. */
AF_API int64_t rn_param_count(int32_t P);

/* Create a generator for P phases (1..65536): parameters, Adam moments and
 * activations on the device, all zero.  stream: a cudaStream_t (NULL =
 * legacy default stream).  Synchronous. */
AF_API af_status rn_create(int32_t P, void* stream, rn_net** out);

/* Free the handle (synchronises its stream first). */
AF_API af_status rn_destroy(rn_net* rn);

/* Message of the last failed call ("" if none); rn may be NULL (the calling
 * thread's last failed rn_create). */
AF_API const char* rn_last_error(const rn_net* rn);

/* Copy rn_param_count(P) parameters from / to the host and, on set, zero the
 * Adam moments.  Synchronous. */
AF_API af_status rn_set_params(rn_net* rn, const float* theta_host);
AF_API af_status rn_get_params(rn_net* rn, float* theta_host);

/* Copy the Adam moments (rn_param_count(P) floats each) from / to the host,
 * for checkpoints; set after rn_set_params, which zeroes them.  Synchronous. */
AF_API af_status rn_set_adam(rn_net* rn, const float* m_host, const float* v_host);
AF_API af_status rn_get_adam(rn_net* rn, float* m_host, float* v_host);

/* u_dev [P] <- f_theta(y0_dev) before the sigmoid. */
AF_API af_status rn_forward(rn_net* rn, const float* y0_dev, float* u_dev);

/* One Adam step (step t >= 1, rate lr) on every parameter with the gradient
 * of a loss whose derivative w.r.t. the output is du_dev [P] (dL/du, at the
 * activations of the last rn_forward / rn_train_step), then u_dev <- the new
 * f_theta(y0_dev). */
AF_API af_status rn_train_step(rn_net* rn, const float* y0_dev, const float* du_dev, float lr, int64_t t,
                               float* u_dev);

/*
 * Make sqngd_step train the generator: Step B of Algorithm 1 then takes, per
 * evaluation, dL/du from the loss (no update of the logits), one Adam step on
 * theta with the context's lr_x, beta1, beta2, adam_eps and its step counter,
 * and the forward pass; st->u_dev holds the generator's output u throughout.
 * Before the first sqngd_step the caller sets st->u_dev = u by rn_forward.
 * y0_dev [P = M N] stays owned by the caller and must outlive the context's
 * use of it.  rn = NULL detaches.  Not combined with trained thresholds.
 */
AF_API af_status sqngd_attach_generator(af_ctx* ctx, rn_net* rn, const float* y0_dev);

#ifdef __cplusplus
}
#endif

#endif
