/*
 * sqngd.h -- C ABI of the SQNGD hot path on one GB300 GPU (sm_103a).
 *
 * The library evaluates every auto- and cross-ambiguity function between M
 * unimodular waveforms x_m and M receive filters h_l over a delay-Doppler
 * grid, the sidelobe + SNR-loss objective of the SQNGD method and its
 * gradient, and runs the quantizers, filter projection and alternating Adam
 * steps of the method's Algorithm 1.
 *
 * Paper: J. Ma, Y. Li, J. Wang, Y. Zhou, "Joint Design of Doppler-Resilient
 * Unimodular Discrete-Phase Waveforms and Receiving Filters for MIMO Radars".
 * Equation numbers below are the paper's.
 *
 * General conventions
 *  - Every entry point has C linkage, never throws, and returns af_status.
 *    On failure af_last_error(ctx) holds a one-line message.
 *  - Pointers named *_dev are DEVICE pointers owned by the caller; *_host are
 *    host pointers owned by the caller.  The context owns only its own
 *    workspace and tables.
 *  - Complex arrays are interleaved float pairs (re, im): a "complex [M][N]"
 *    array holds 2*M*N floats, element (m, n) at index 2*(m*N + n).
 *  - Waveform/filter layout is [M][N] row-major (waveform-major, the vec of
 *    the paper's N x M matrices, Eq. 16).
 *  - The ambiguity grid is [M][M][D][L]: pair (m, l) = (transmit waveform m,
 *    receive filter l), delay index d = k - k_lo (D = k_hi - k_lo + 1),
 *    Doppler bin j.  The "linear cell index" is ((m*M + l)*D + d)*L + j.
 *  - Work is enqueued on the context's stream (the one given to af_init) and
 *    is asynchronous unless the entry point says otherwise; device outputs
 *    are valid once that stream has been synchronised (af_sync).
 *  - A context is not thread-safe; use one context per stream.
 *  - Sample index n runs 0..N-1 (the paper counts from 1, which multiplies
 *    every chi by a unimodular factor and changes no |chi|, loss or gradient).
 *  - Doppler nu is in cycles per chip: the paper's normalised f (cycles per
 *    waveform, Eq. 6) is f = nu * N.
 */
#ifndef SQNGD_H
#define SQNGD_H

#include <stdint.h>

#if defined(__GNUC__)
#define AF_API __attribute__((visibility("default")))
#else
#define AF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AF_OK = 0,
    AF_ERR_INVALID_ARG = 1,   /* bad size, range or pointer; nothing was launched */
    AF_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has the CUDA error) */
    AF_ERR_NONFINITE = 3,     /* a loss or gradient came out NaN/Inf (reported by af_sync) */
    AF_ERR_TIMEOUT = 4,       /* a bounded device-side pipeline wait (AF_PATH_SPLIT_BF16)
                                 gave up; the kernel ended cleanly (reported by af_sync) */
    AF_ERR_OOM = 5,           /* workspace allocation failed */
    AF_ERR_UNIMPLEMENTED = 6  /* the requested path does not support this configuration */
} af_status;

/* Evaluation path for the Doppler transform of each delay row. */
enum {
    AF_PATH_AUTO = 0,        /* FFT when the grid is uniform with spacing 1/L, else DFT */
    AF_PATH_FFT = 1,         /* FP32 shared-memory FFT; grid nu_j = nu_0 + j/L, L = 2^p, 32..4096 */
    AF_PATH_DFT = 2,         /* FP32 direct DFT (any grid); SIMT */
    AF_PATH_SPLIT_BF16 = 3   /* the same direct DFT of Eq. 6 as a real-embedded GEMM on
                                tcgen05 tensor cores, both operands split into BF16
                                hi + lo (three products), FP32 accumulation; any grid,
                                meant for narrow Doppler windows; pnorm must be 0 */
};

/* Number of doubles in a terms record (followed by M values of p_m). */
#define AF_TERMS_FIXED 8

typedef struct af_ctx af_ctx;

/*
 * Problem and optimiser configuration.  Inputs of Algorithm 1 plus the
 * hyper-parameters of Section IV.
 */
typedef struct af_config {
    int32_t M;               /* waveforms = receive filters, 1..16 */
    int32_t N;               /* chips per waveform, 2..4096 */
    int32_t B;               /* phase alphabet size (Eq. 5), 2..1024 */
    int32_t L;               /* Doppler bins, 1..4096 */
    const double* nu;        /* host [L]: Doppler grid, cycles/chip, copied at af_init */
    int32_t k_lo, k_hi;      /* delay window, -(N-1) <= k_lo <= k_hi <= N-1 */
    const float* weights;    /* host [D][L] ROI weights w(tau, f) >= 0 (Eqs. 8-9), copied;
                                NULL means w = 1/N on every cell of the grid */
    double eps;              /* epsilon of Eq. 42, in [0, 1] */
    double snrl_db;          /* target SNRL mu~ in dB (Eq. 39), >= 0 */
    int32_t r_n;             /* copies of the soft quantizer (Eq. 24), >= 1 */
    double c;                /* tanh sharpness c (Eq. 24), > 0 */
    double pnorm;            /* 0: exact max of Eqs. 7-9 (the paper's loss);
                                > 0: smooth p-norm (sum (w|chi|)^p)^(1/p) per class
                                (an extension; needs p >= 1) */
    int32_t path;            /* AF_PATH_* */
    int32_t n_h, n_x;        /* inner Adam steps on H and on the transmit logits (Alg. 1) */
    double lr_h, lr_x;       /* Adam learning rates (eta_h, eta_x) */
    double beta1, beta2, adam_eps;  /* Adam constants; 0 selects 0.9, 0.999, 1e-8 */
    int32_t matched;         /* 0: joint design (SQNGD).  1: SQNAF (Section IV): every
                                receive filter is its waveform, h_m = x_m, so there is no
                                filter to optimise (needs n_h = 0); losses and gradients
                                are those of L(x, x) and filter arguments are ignored */
    int32_t train_rho;       /* 0: thresholds fixed.  1: the rho_i of Eq. 24 are trained in Step B
                                (Section III-C): Adam on dL/drho with lr_rho after each transmit
                                step, then the projection of af_project_thresholds.  Needs
                                K = B r_n <= 8192 */
    double lr_rho;           /* Adam learning rate of the thresholds, >= 0 */
} af_config;

/*
 * Optimiser state for sqngd_step, all device buffers owned by the caller.
 * The transmit parameters are direct logits u: z = sigmoid(u) in [0, 1] is
 * the continuous phase that the quantizers of Eqs. 24 and 43 act on.
 */
typedef struct af_state {
    float* u_dev;            /* [M][N] logits */
    float* h_dev;            /* complex [M][N] receive filters (H_Re + j H_Im, Eq. 28) */
    float* m_u_dev;          /* [M][N] Adam first moment of u  (zero-initialised by caller) */
    float* v_u_dev;          /* [M][N] Adam second moment of u */
    float* m_h_dev;          /* [M][2N] Adam first moment of (H_Re, H_Im), interleaved */
    float* v_h_dev;          /* [M][2N] Adam second moment */
    int32_t* best_q_dev;     /* [M][N] hard indices q of the best design so far (may be NULL) */
    float* best_h_dev;       /* complex [M][N] filters of the best design (may be NULL) */
    double* best_dev;        /* [4]: best hard L_WPSL, its loss, its outer iteration, its max
                                SNRL dB; caller initialises [0] to +inf */
    int64_t t_h, t_x;        /* Adam step counters (host side, advanced by sqngd_step) */
    int64_t outer;           /* outer iterations done (host side, advanced by sqngd_step) */
} af_state;

/* Create a context: validates cfg, copies the grid, weights and thresholds
 * rho_i = (i + 1/2)/K (K = B r_n, Eq. 24) to the device, builds twiddle and
 * phase tables in FP64 on the host, allocates the workspace.  stream is a
 * cudaStream_t (NULL = legacy default stream).  Synchronous. */
AF_API af_status af_init(const af_config* cfg, void* stream, af_ctx** out);

/* Free the context and its workspace (synchronises its stream first). */
AF_API af_status af_destroy(af_ctx* ctx);

/* Message of the last failed call on ctx ("" if none).  ctx may be NULL, in
 * which case the message of the calling thread's last failed call that has
 * no context (af_init, af_loss_terms_noalloc) is returned. */
AF_API const char* af_last_error(const af_ctx* ctx);

/* Path the context resolved to (AF_PATH_FFT, AF_PATH_DFT or AF_PATH_SPLIT_BF16). */
AF_API int32_t af_path_of(const af_ctx* ctx);

/* Wait for the context's stream; returns AF_ERR_NONFINITE if any loss or
 * gradient since the last af_sync was NaN/Inf, AF_ERR_TIMEOUT if a
 * tensor-core pipeline wait gave up, AF_ERR_CUDA on a CUDA error. */
AF_API af_status af_sync(af_ctx* ctx);

/* Replace the quantization thresholds (host [K] floats, strictly increasing
 * inside [0, 1]; Section III-C keeps them ordered).  Synchronous. */
AF_API af_status af_set_thresholds(af_ctx* ctx, const float* rho_host);

/*
 * Eq. 6 on the whole grid: chi_dev receives complex [M][M][D][L] (FP32).
 * x_dev, h_dev: complex [M][N].  The materialising variant of the forward
 * pass (the loss path never stores chi).
 */
AF_API af_status af_ambiguity(af_ctx* ctx, const float* x_dev, const float* h_dev, float* chi_dev);

/*
 * The fused forward pass alone (lag products, Doppler transform and the
 * per-CTA sidelobe partials of Eqs. 7-9 into the context's workspace, plus
 * A_mm(0,0) of Eq. 38), without loss assembly or gradient.  For timing the
 * dominant kernel in isolation; af_loss_grad_xh runs the same pass first.
 */
AF_API af_status af_forward(af_ctx* ctx, const float* x_dev, const float* h_dev);

/*
 * Loss (Eq. 42 with Eqs. 7-9, 37, 38, 41) and its gradient for given complex
 * waveforms x and filters h.
 *  terms_dev: device [AF_TERMS_FIXED + M] doubles: [0] L, [1] L_WPSL,
 *     [2] WAPSL, [3] WCPSL, [4] L_SNRL, [5] winning class (0 auto, 1 cross),
 *     [6] argmax cell of the auto class, [7] of the cross class (linear cell
 *     index, -1 if the class is empty), then p_m for m = 0..M-1 (Eq. 38).
 *     May be NULL.
 *  grad_x_dev, grad_h_dev: complex [M][N]: dL/dRe + j dL/dIm; may be NULL.
 * The exact max is differentiated at one cell per class: the largest
 * w^2|chi|^2 in FP32, ties to the lowest linear cell index; WAPSL wins a tie
 * with WCPSL.
 * Matched contexts (cfg.matched = 1): h_dev is ignored (may be NULL), the
 * loss is L(x, x), grad_x_dev receives its total gradient (the sum of the
 * transmit and filter partials at h = x) and grad_h_dev must be NULL.
 * With both gradient outputs NULL the p-norm loss skips its dense adjoint
 * (the loss terms alone are computed).
 */
AF_API af_status af_loss_grad_xh(af_ctx* ctx, const float* x_dev, const float* h_dev,
                          double* terms_dev, float* grad_x_dev, float* grad_h_dev);

/*
 * Loss and gradient through the transmit chain of Section III-A:
 * z = sigmoid(u), y = Q_A(z) (Eq. 24), x = e^{j 2 pi y} (Eq. 23) when
 * use_hard = 0; the hard waveform of Eq. 43 (no gradient to u) when
 * use_hard = 1.  u_dev: [M][N]; h_dev complex [M][N];
 * grad_u_dev: [M][N] (ignored when use_hard = 1), grad_h_dev complex [M][N];
 * terms_dev as in af_loss_grad_xh.  Any output may be NULL; with no
 * gradient output the p-norm loss skips its dense adjoint.
 * Matched contexts: h_dev is ignored (may be NULL), grad_u_dev is the
 * gradient of L(x, x) and grad_h_dev must be NULL.
 */
AF_API af_status af_loss_grad(af_ctx* ctx, const float* u_dev, const float* h_dev, int32_t use_hard,
                       double* terms_dev, float* grad_u_dev, float* grad_h_dev);

/*
 * Hard quantizer (Eq. 43, c -> infinity reading): q = #{i : rho_i <= z},
 * phase index b = q mod B, x_hard = e^{j 2 pi b / B} from an FP64-built table.
 * z_dev: [n] continuous phases in [0, 1]; q_dev: [n] int32 (may be NULL);
 * x_dev: complex [n] (may be NULL).  n <= M*N is not required.
 */
AF_API af_status quantize(af_ctx* ctx, const float* z_dev, int64_t n, int32_t* q_dev, float* x_dev);

/*
 * Soft quantizer (Eq. 24) on continuous phases: y = Q_A(z), dydz = Q_A'(z),
 * x = e^{j 2 pi y}.  Any output may be NULL.
 */
AF_API af_status soft_quantize(af_ctx* ctx, const float* z_dev, int64_t n, float* y_dev,
                        float* dydz_dev, float* x_dev);

/*
 * Loss and gradients through the soft transmit chain, as af_loss_grad with
 * use_hard = 0, plus grad_rho_dev: [K] floats, dL/drho_i of Eq. 24 with the
 * context's current thresholds (Section III-C):
 *   sum over elements e of dL/dy_e * (-a c (1 - tanh^2(c (z_e - rho_i)))),
 * accumulated in a fixed-point sum whose value does not depend on the order
 * of accumulation.  Needs K <= 8192.  grad_u_dev, grad_h_dev may be NULL.
 */
AF_API af_status af_loss_grad_rho(af_ctx* ctx, const float* u_dev, const float* h_dev, double* terms_dev,
                                  float* grad_u_dev, float* grad_h_dev, float* grad_rho_dev);

/* Copy the context's K thresholds (host [K] floats).  Synchronous. */
AF_API af_status af_get_thresholds(af_ctx* ctx, float* rho_host);

/*
 * Projection of K thresholds (device [K] floats, in place) onto the nearest
 * ordered set 0 <= rho_0 <= ... <= rho_{K-1} <= 1 in the Euclidean sense
 * (isotonic regression by pooling adjacent violators, then clipping): the
 * ordering that Section III-C requires of the thresholds.  Needs K <= 8192.
 */
AF_API af_status af_project_thresholds(af_ctx* ctx, float* rho_dev);

/* Energy projection of Eq. 32 in place: h_m <- sqrt(N/||h_m||^2) h_m, norms
 * accumulated in FP64.  h_dev complex [M][N]. */
AF_API af_status af_project(af_ctx* ctx, float* h_dev);

/*
 * Initialisation of Algorithm 1 from drawn phase indices b (Eq. 29):
 * u = logit(z0) with z0 = (floor(r_n/2) B + b)/K (the middle copy, so the
 * hard quantizer returns b), h = x0 + noise, projected (Eq. 32).  The filters
 * start matched to the waveforms under Eq. 6's x h^* convention.
 * b_dev: [M][N] int32 in [0, B); noise_dev: complex [M][N] or NULL.
 */
AF_API af_status sqngd_init(af_ctx* ctx, const int32_t* b_dev, const float* noise_dev,
                     float* u_dev, float* h_dev);

/*
 * n_outer outer iterations of Algorithm 1: X_hard from u; n_h x {loss and
 * grad_H at X_hard; Adam on (H_Re, H_Im); projection (Eq. 32)}; n_x x {X_soft
 * from u; loss and grad_u; Adam on u}.  Precision inside the step: the
 * products and transforms in FP32; A_mm(0,0) and the projection norms
 * ||h_m||^2 as double-float sums of exact FP32 products (about 44
 * significant bits); p_m, L_SNRL, the SNRL gradient coefficient and the
 * loss assembly in FP64; the projection's scale factor in FP32 (below the
 * FP32 rounding of the stored taps).  One outer iteration is replayed as a
 * CUDA graph.  The first evaluation of every outer iteration scores the
 * current hard design; the best one (lowest L_WPSL among designs whose max
 * SNRL is within 0.05 dB of the target) is copied to best_q/best_h.
 * log_host: if not NULL, receives [n_outer][n_h + n_x][4] doubles (L, L_WPSL,
 * L_SNRL, winning class) and the call synchronises; otherwise it is
 * asynchronous.  Advances st->t_h, st->t_x, st->outer.
 * Matched contexts (SQNAF): Step A is skipped and h_dev, m_h_dev, v_h_dev are
 * not touched (they may be NULL); each outer iteration scores the hard design
 * L(X_hard, X_hard) for the best-design record, then runs the n_x transmit
 * steps on L(X_soft, X_soft); best_h receives X_hard of the best design and
 * the log has 1 + n_x evaluations per outer iteration (the score first).
 */
AF_API af_status sqngd_step(af_ctx* ctx, af_state* st, int32_t n_outer, double* log_host);

/* Record of the stopping rule, kept by the caller between calls (and in
 * checkpoints) so that a resumed run applies the rule as an uninterrupted one. */
typedef struct af_stop {
    double best_wpsl;        /* lowest hard L_WPSL scored so far; +inf before the first */
    int64_t best_outer;      /* outer iteration (st->outer numbering) that scored it; a negative
                                value (a fresh record) is set to st->outer - 1 by sqngd_run */
    int32_t stopped;         /* out: 0 not stopped, 1 the patience rule fired, 2 t_max reached */
} af_stop;

/*
 * Algorithm 1 with its stopping test (Section III-C): training ends when
 * further outer iterations bring no improvement in the WPSL, or when the
 * maximum number T of outer iterations is reached.  Reading: the WPSL is
 * the hard design's L_WPSL, scored by the first evaluation of every outer
 * iteration (the Step-A evaluation at X_hard, or the hard-design score of a
 * matched context); an outer iteration improves when that value is strictly
 * below stop->best_wpsl; the run stops after outer iteration t as soon as
 * t - stop->best_outer >= patience, or once st->outer reaches t_max.
 * The iterations run through sqngd_step in chunks sized so that the rule can
 * fire only at a chunk's last iteration, so the stop is exact (no iteration
 * beyond it runs) and the results equal those of sqngd_step over the same
 * number of iterations.  Each chunk's log is read back (synchronous call).
 * log_host: NULL, or room for [t_max - st->outer][evals][4] doubles as in
 * sqngd_step, of which the first *n_done rows are written.  patience >= 1.
 * Needs a hard evaluation in every outer iteration: n_h >= 1, or matched.
 */
AF_API af_status sqngd_run(af_ctx* ctx, af_state* st, int64_t t_max, int32_t patience, af_stop* stop,
                           double* log_host, int64_t* n_done);

/*
 * The quantization thresholds' state, for checkpoints: rho [K], their Adam
 * moments m_rho, v_rho [K] (zero unless cfg.train_rho), and `uniform`: 1 when
 * the quantizers use the default set rho_i = (i + 1/2)/K computed by
 * arithmetic, 0 when they read the table (user-set or trained thresholds).
 * Host buffers; m_host, v_host may be NULL.  Synchronous.  The setter
 * accepts any non-decreasing rho in [0, 1]; uniform = 1 requires rho to be
 * the default set.
 */
AF_API af_status af_get_rho_state(af_ctx* ctx, float* rho_host, float* m_host, float* v_host, int32_t* uniform);
AF_API af_status af_set_rho_state(af_ctx* ctx, const float* rho_host, const float* m_host, const float* v_host,
                                  int32_t uniform);

/*
 * Acceptance metrics in FP64 on the GPU (Eq. 48 and Eq. 10) for the hard
 * design of logits u and filters h: out_host[0] APSL dB, [1] CPSL dB,
 * [2] PSLR dB = max of the two, [3] max_m SNRL dB, then SNRL dB for each m.
 * PSL is max |chi| over the ROI (cells of positive weight; the auto term
 * skips tau = 0).  out_host: [4 + M] doubles.  Synchronous.
 * Matched contexts: h_dev is ignored (may be NULL); the filters are the hard
 * waveforms.
 */
AF_API af_status af_eval_hard(af_ctx* ctx, const float* u_dev, const float* h_dev, double* out_host);

/*
 * Loss terms without any device allocation.  The paper has no counterpart:
 * this is a service entry point for callers that cannot call cudaMalloc --
 * code running while a stream is captured into a CUDA graph, hosts whose
 * framework owns the device memory pool and forbids raw allocations, and
 * latency-critical loops that cannot afford an allocation's implicit
 * synchronisation.  It needs no context.
 *
 * Computes the same terms record as af_loss_grad_xh (terms_dev: device
 * [AF_TERMS_FIXED + M] doubles) for waveforms x_dev and filters h_dev
 * (complex [M][N], device) on the uniform Doppler grid nu_j = nu0 + j/L
 * (cycles/chip), delays k_lo..k_hi, weight 1/N on every cell, loss constants
 * eps and snrl_db; no gradient.  Enqueued on `stream` (a cudaStream_t).
 *
 * All scratch lives in one file-scope device array of about 0.3 MB that
 * every GPU loading the library keeps until exit.  Limits: M <= 16,
 * N <= 4096, L a power of two in 32..4096, and the forward pass must fit in
 * shared memory; anything else returns AF_ERR_INVALID_ARG before any launch.
 * The first call on a device looks the array up (cudaGetSymbolAddress):
 * make it before any stream capture.  Calls share the array, so calls that
 * overlap on the GPU race; every call rewrites the scratch it reads, so
 * nothing needs clearing between calls.  Returns AF_ERR_CUDA if a lookup or
 * launch fails.  On any failure af_last_error(NULL), called from the same
 * thread, gives the reason.
 */
AF_API af_status af_loss_terms_noalloc(int32_t M, int32_t N, int32_t L, double nu0, int32_t k_lo, int32_t k_hi,
                                       double eps, double snrl_db, const float* x_dev, const float* h_dev,
                                       double* terms_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SQNGD_H */
