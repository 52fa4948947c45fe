/*
 * warmstart.h -- C ABI of the learned warm-start network.
 *
 * The paper generates the continuous transmit phases with a network whose
 * input is the initial phase configuration y0 (Section II-B, Eq. 17); this
 * library optimises direct logits instead and uses the network below only
 * to propose the initial code.  The network is not in the paper.
 *
 * Network (all sizes fixed): input features F[32][N] of one design --
 *   c = 0        n / N
 *   c = 1+2i,2+2i  cos, sin of 2 pi f_i n / N, f_i = 1, 2, 4, 8
 *   c = 9..13    the five conditioning scalars cond[0..4], broadcast
 *   c = 14+2m, 15+2m  cos, sin of 2 pi b0[m][n] / B (m < M; 0 otherwise)
 *   c = 22..31   0
 * four 1-D convolutions of width 5 with zero padding 2 (32 -> 64 -> 64 ->
 * 64 -> 64 channels), tanh after the first three; output channel
 * m * 16 + q is the logit of phase level q of waveform m.  Requires M <= 4,
 * B <= 16.  Weights are stored in FP16, biases in FP32, accumulation is FP32.
 *
 * Parameters are exchanged as one FP32 vector in the order
 * [W1 (64x32x5), b1 (64), W2 (64x64x5), b2, W3, b3, W4, b4], W[co][ci][t]
 * row-major; the forward pass uses the FP16 images (round to nearest even)
 * of the W parts.
 *
 * Training loss: mean over the batch of the per-design cross-entropy
 * mean_{m<M, n<N} -log softmax_{q<B}(logits[m*16+q][n])[target[m][n]];
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias corrected) on FP32 master
 * parameters.
 *
 * Device arrays are caller-owned; layouts are row-major with the batch index
 * outermost.  Work is enqueued on the stream given at ws_create; every
 * entry point returns a status (the af_status codes of sqngd.h).
 */
#ifndef SQNGD_WARMSTART_H
#define SQNGD_WARMSTART_H

#include <stdint.h>

#include "sqngd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ws_net ws_net;

/* Configuration shared by every design of a batch. */
typedef struct ws_config {
    int32_t M;        /* waveforms, 1..4 */
    int32_t N;        /* chips, 1..n_max */
    int32_t B;        /* phase levels, 2..16 */
    double cond[5];   /* conditioning scalars (features 9..13) */
} ws_config;

/* Number of parameters (FP32 vector length). */
AF_API int64_t ws_param_count(void);

/* Allocate the weights, Adam state and the activations of batch_max designs
 * of at most n_max chips; parameters start at 0 (call ws_set_params).
 * stream: a cudaStream_t (NULL = legacy default stream). */
AF_API af_status ws_create(int32_t batch_max, int32_t n_max, void* stream, ws_net** out);
AF_API af_status ws_destroy(ws_net* net);
AF_API const char* ws_last_error(const ws_net* net);

/* Host FP32 parameter vector in / out (synchronous).  Setting resets the
 * Adam moments and step counter. */
AF_API af_status ws_set_params(ws_net* net, const float* params_host);
AF_API af_status ws_get_params(ws_net* net, float* params_host);

/* Forward pass of `batch` designs with initial codes b0_dev ([batch][M][N]
 * int32 in [0, B)).  logits_dev: [batch][64][N] FP32 or NULL; b_dev:
 * [batch][M][N] int32 argmax over q < B (lowest q on ties) or NULL.
 * Asynchronous. */
AF_API af_status ws_forward(ws_net* net, const ws_config* cfg, int32_t batch, const int32_t* b0_dev,
                            float* logits_dev, int32_t* b_dev);

/* Loss and gradient of a batch without updating the parameters
 * (synchronous): loss_host (may be NULL), grad_host [ws_param_count()] FP32
 * in the parameter order (may be NULL). */
AF_API af_status ws_loss_grad(ws_net* net, const ws_config* cfg, int32_t batch, const int32_t* b0_dev,
                              const int32_t* target_dev, double* loss_host, float* grad_host);

/* One Adam step on a batch with learning rate lr.  loss_host: if not NULL
 * receives the batch loss before the step and the call synchronises;
 * otherwise it is asynchronous. */
AF_API af_status ws_train_step(ws_net* net, const ws_config* cfg, int32_t batch, const int32_t* b0_dev,
                               const int32_t* target_dev, float lr, double* loss_host);

#ifdef __cplusplus
}
#endif

#endif
