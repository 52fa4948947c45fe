// af_step.cuh -- argument blocks of the per-step kernels (host + device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace af {

// Transmit-chain constants (Eq. 24 with K = B r_n thresholds).
struct QuantArgs {
    const float* rho;     // [K] sorted thresholds
    int K, B;
    float a, c;           // a = 1/(2B), sharpness c
    float win;            // half window (in z units) outside which tanh is +-1 in FP32
    const float2* level;  // [B] e^{j 2 pi b / B}, FP64-built
    int uniform;          // rho_i = (i + 1/2)/K: indices can be found arithmetically
};

enum FinMode : int {
    FIN_GRAD_XH = 0,   // write grad_x, grad_h
    FIN_GRAD_U = 1,    // write grad_u (soft chain) and grad_h
    FIN_ADAM_H = 2,    // Adam on (H_Re, H_Im) + projection (Step A)
    FIN_ADAM_U = 3,    // Adam on u (Step B)
    FIN_SCORE = 4      // loss and best-design record only (SQNAF's score of the hard design)
};

enum NextWave : int { NEXT_NONE = 0, NEXT_SOFT = 1, NEXT_HARD = 2 };

struct FinArgs {
    int M, N, L, D, k_lo;
    int nblk, ctas_per_pair;
    const float* pkey;
    const long long* pidx;
    const float* pvmax;
    const float* psum;
    const float2* pchi;       // [nblk] chi at each forward CTA's best cell
    const double2* cdiag;     // [M]
    int weight_mode;          // WeightMode
    float w0;
    const float* wmap;        // [D][L]
    double eps, ptar;
    double snrl_coef;         // (1 - eps) (2 / M) / N: G_m = snrl_coef (p_m - p_tar) c_m / |c_m|
    double inv_N;             // 1/N
    int pdl;                  // launch with programmatic stream serialisation
    float half_p;             // p/2 (0 = exact max)
    int grid_fft;             // 1: nu_j = nu_0 + j/L (phasor = pre(n) wL[(j n) mod L]); 0: table E
    const float2* pre;        // [N]
    const float2* wL;         // [L] e^{j 2 pi i / L}
    const float2* E;          // [N][L] e^{j 2 pi nu_j n}
    const float2* dense_g;    // [nblk_dense][2][M*N] partial sidelobe gradients (p-norm) or null
    int n_dense;              // number of dense partial blocks
    // waveforms used by this evaluation
    const float2* x;          // [M][N] waveforms of this evaluation
    const float* dydz;        // [M][N] Q_A'(z) of this evaluation (soft chain)
    float2* x_next;           // [M][N] waveform written for the next evaluation
    float* dydz_next;         // [M][N] its Q_A'(z) (soft)
    const float2* h_in;       // [M][N] filters of this evaluation
    // outputs
    int mode;                 // FinMode
    double* terms;            // [8 + M] or null
    double* log;              // base of the log or null; slot = (ctr[0]-1)*evals + eval
    int evals_per_outer, eval_index;
    int* err_flag;
    float2* grad_x;
    float2* grad_h;
    float* grad_u;
    // optimiser state (sqngd_step)
    float* u;                 // [M][N] logits
    float2* h;                // [M][N] filters (updated in place in FIN_ADAM_H)
    float2* m_h;
    float2* v_h;
    float* m_u;
    float* v_u;
    float lr, b1, b2, adam_eps;
    const long long* ctr;     // device [4]: outer iteration (1-based within the call), t_h0, t_x0, outer0
    int inner;                // inner step index within Step A or Step B
    int n_h, n_x;             // inner steps per outer iteration
    int next_wave;            // NextWave
    QuantArgs qa;
    // best-design tracking (first Step-A evaluation of an outer iteration)
    int snap_best;
    double* best2;            // [2][4] ping-pong records
    int32_t* best_q;
    float2* best_h;
    double snrl_db;
    double p_accept2;         // (10^{-(snrl_db + 0.05)/20})^2: a design is acceptable when min p_m^2 >= this
    int matched;              // SQNAF: h = x, the gradient of x is the sum of both partials
    float* gy_out;            // [M][N] dL/dy and the z it was taken at (trainable thresholds), or null
    float* z_out;
    float* du_out;            // FIN_ADAM_U: [M][N] dL/du written instead of the Adam step (generator), or null
    // FP32 copy of eps (the sparse gradient coefficient), filled by launch_fin
    float eps_f;
};

enum RhoMode : int {
    RHO_GRAD = 0,      // write dL/drho only
    RHO_STEP = 1,      // dL/drho, Adam on rho, projection
    RHO_PROJECT = 2    // projection of rho in place
};

struct RhoArgs {
    int mode;                 // RhoMode
    int n;                    // elements M*N
    const float* gy;          // [n] dL/dy of the evaluation
    const float* z;           // [n] z of the evaluation's soft waveform
    QuantArgs q;              // thresholds (q.rho = the trained table), a, c, window
    float* rho;               // [K] thresholds, updated in place (RHO_STEP, RHO_PROJECT)
    long long* acc;           // [K] fixed-point gradient accumulator, left zeroed
    float* grad_out;          // [K] dL/drho (RHO_GRAD)
    float* m_rho;             // [K] Adam moments
    float* v_rho;
    float lr, b1, b2, adam_eps;
    const long long* ctr;     // step counters (as FinArgs::ctr)
    int inner, n_x;           // Step-B index and steps per outer iteration
    int pdl;
};

struct AccArgs {
    int M, N, nblk, ctas_per_pair;
    const double* pkey;
    const double2* cdiag;
    const double2* x;
    const double2* h;
    double* out;              // [4 + M]
};

}  // namespace af
