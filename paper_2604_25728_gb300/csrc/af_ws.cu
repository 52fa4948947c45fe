// af_ws.cu -- the learned warm-start network: features, four 1-D
// convolutions (FP16 weights, FP32 accumulation), softmax cross-entropy,
// backward pass, Adam, argmax inference, and its C ABI (warmstart.h).
//
// Activations are [design][channel][n] FP32.  A convolution block computes
// all 64 output channels of 64 consecutive positions of one design: the
// input tile (with a 2-position halo on each side) and the layer's FP16
// weights sit in shared memory, each thread accumulates 4 channels x 4
// positions.  The input gradient is the same convolution with the weights
// transposed and flipped in t, fused with the tanh derivative.  Weight
// gradients reduce over (design, position) in fixed-order splits, then a
// second kernel sums the splits in order (deterministic).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/warmstart.h"

namespace ws {

constexpr int CIN = 32, CH = 64, KW = 5, PAD = 2, QMAX = 16, MMAX = 4;
constexpr int TN = 64;                 // positions per convolution block
constexpr int kThreads = 256;
constexpr int kSplits = 16;            // weight-gradient splits over (design, position) tiles

constexpr long long wsize(int l) { return (long long)CH * (l == 0 ? CIN : CH) * KW; }
constexpr long long woff(int l) {      // offset of W_l in the packed parameter vector
    return l == 0 ? 0 : woff(l - 1) + wsize(l - 1) + CH;
}
constexpr long long boff(int l) { return woff(l) + wsize(l); }
constexpr long long kParams = woff(4);

enum ConvMode : int { FWD_TANH = 0, FWD_LINEAR = 1, BWD_DATA = 2 };

// ---------------------------------------------------------------- features --
__global__ void features_kernel(const int32_t* b0, int M, int N, int B, float c0, float c1, float c2, float c3,
                                float c4, float* F, int batch) {
    const long long total = (long long)batch * CIN * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e % N);
        const int c = (int)((e / N) % CIN);
        const int d = (int)(e / ((long long)N * CIN));
        float v = 0.f;
        if (c == 0) {
            v = (float)n / (float)N;
        } else if (c <= 8) {
            const int i = (c - 1) / 2;
            const float f = (float)(1 << i);
            float s, co;
            sincospif(2.f * f * (float)n / (float)N, &s, &co);
            v = (c & 1) ? co : s;
        } else if (c <= 13) {
            const float cc[5] = {c0, c1, c2, c3, c4};
            v = cc[c - 9];
        } else if (c <= 21) {
            const int m = (c - 14) / 2;
            if (m < M) {
                const int b = b0[((long long)d * M + m) * N + n];
                float s, co;
                sincospif(2.f * (float)b / (float)B, &s, &co);
                v = (c & 1) ? s : co;
            }
        }
        F[e] = v;
    }
}

// ------------------------------------------------------------- convolution --
// FWD_*:    out[d][co][n] = bias[co] + sum_ci sum_t W[co][ci][t] in[d][ci][n + t - 2]  (then tanh)
// BWD_DATA: out[d][ci][n] = (1 - act[d][ci][n]^2) sum_co sum_t W[co][ci][t] in[d][co][n - t + 2]
// (in = dL/dz of the layer, act = the layer's input activation).
template <int CI, int MODE>
__global__ void __launch_bounds__(kThreads) conv_kernel(const float* in, const __half* W, const float* bias,
                                                        const float* act, float* out, int N) {
    extern __shared__ __align__(16) unsigned char smem[];
    __half* ws_ = reinterpret_cast<__half*>(smem);                       // [64][CI][5] in the kernel's order
    float* xt = reinterpret_cast<float*>(smem + sizeof(__half) * CH * CI * KW);   // [CI][TN + 4]
    const int d = blockIdx.y;
    const int n0 = blockIdx.x * TN;
    const int tid = threadIdx.x;
    // weights: wk[o][i][t] = W[o][i][t] (forward) or W[i][o][4 - t] (input gradient)
    for (int e = tid; e < CH * CI * KW; e += kThreads) {
        const int t = e % KW, i = (e / KW) % CI, o = e / (KW * CI);
        ws_[e] = (MODE == BWD_DATA) ? W[((long long)i * CH + o) * KW + (KW - 1 - t)] : W[e];
    }
    const float* src = in + (long long)d * CI * N;
    for (int e = tid; e < CI * (TN + 4); e += kThreads) {
        const int i = e / (TN + 4), j = e % (TN + 4);
        const int p = n0 + j - PAD;
        xt[e] = (p >= 0 && p < N) ? src[(long long)i * N + p] : 0.f;
    }
    __syncthreads();
    const int ty = tid / 16, tx = tid % 16;     // channels ty*4 .. +3, positions tx + 16 j
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[a][j] = 0.f;
    for (int i = 0; i < CI; ++i) {
        const float* xr = xt + i * (TN + 4);
#pragma unroll
        for (int t = 0; t < KW; ++t) {
            float w[4], x[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) w[a] = __half2float(ws_[((ty * 4 + a) * CI + i) * KW + t]);
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = xr[tx + 16 * j + t];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[a][j] = fmaf(w[a], x[j], acc[a][j]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int o = ty * 4 + a;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            const long long idx = ((long long)d * CH + o) * N + n;
            float v = acc[a][j];
            if (MODE == BWD_DATA) {
                const float y = act[idx];
                v *= (1.f - y * y);
            } else {
                v += bias[o];
                if (MODE == FWD_TANH) v = tanhf(v);
            }
            out[idx] = v;
        }
    }
}

template <int CI, int MODE>
static int conv_smem() { return (int)(sizeof(__half) * CH * CI * KW + sizeof(float) * CI * (TN + 4)); }

template <int CI, int MODE>
static cudaError_t launch_conv(const float* in, const __half* W, const float* bias, const float* act, float* out,
                               int N, int batch, cudaStream_t s) {
    const int smem = conv_smem<CI, MODE>();
    cudaError_t e = cudaFuncSetAttribute(conv_kernel<CI, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((N + TN - 1) / TN, batch);
    conv_kernel<CI, MODE><<<grid, kThreads, smem, s>>>(in, W, bias, act, out, N);
    return cudaGetLastError();
}

// --------------------------------------------------------- weight gradient --
// part[s][co][e], e = ci * 5 + t (< CI * 5) and e = CI * 5 for the bias:
// sum over the (design, position) tiles of split s of g[d][co][n] x[d][ci][n + t - 2].
template <int CI>
__global__ void __launch_bounds__(CI * KW + 32) wgrad_kernel(const float* g, const float* x, float* part, int N,
                                                             int batch) {
    __shared__ float gs[TN];
    __shared__ float xs[CI * (TN + 4)];
    const int co = blockIdx.x, s = blockIdx.y;
    const int tid = threadIdx.x;
    const int tiles_per_design = (N + TN - 1) / TN;
    const int n_tiles = batch * tiles_per_design;
    const int per = (n_tiles + kSplits - 1) / kSplits;
    const int ci = tid / KW, t = tid % KW;
    float acc = 0.f;
    for (int tile = s * per; tile < min(n_tiles, (s + 1) * per); ++tile) {
        const int d = tile / tiles_per_design;
        const int n0 = (tile % tiles_per_design) * TN;
        __syncthreads();
        for (int j = tid; j < TN; j += blockDim.x) {
            const int n = n0 + j;
            gs[j] = (n < N) ? g[((long long)d * CH + co) * N + n] : 0.f;
        }
        for (int e = tid; e < CI * (TN + 4); e += blockDim.x) {
            const int i = e / (TN + 4), j = e % (TN + 4);
            const int p = n0 + j - PAD;
            xs[e] = (p >= 0 && p < N) ? x[((long long)d * CI + i) * N + p] : 0.f;
        }
        __syncthreads();
        if (tid < CI * KW) {
            const float* xr = xs + ci * (TN + 4) + t;
#pragma unroll 8
            for (int j = 0; j < TN; ++j) acc = fmaf(gs[j], xr[j], acc);
        } else if (tid == CI * KW) {
            for (int j = 0; j < TN; ++j) acc += gs[j];
        }
    }
    if (tid <= CI * KW) part[((long long)s * CH + co) * (CI * KW + 1) + tid] = acc;
}

// grad[W_l][co][e] and grad[b_l][co] = sum over splits, in split order.
__global__ void wgrad_reduce_kernel(const float* part, int ci_count, float* gW, float* gb) {
    const int E = ci_count * KW + 1;
    const int total = CH * E;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < kSplits; ++s) acc += part[(long long)s * total + e];
        const int co = e / E, k = e % E;
        if (k < ci_count * KW) gW[co * ci_count * KW + k] = acc;
        else gb[co] = acc;
    }
}

// ----------------------------------------------------------- cross-entropy --
// g[d][c][n] = (softmax - onehot) / (M N batch) for c = m*16 + q, q < B, m < M; 0 otherwise.
// lpart[block] = sum of the block's -log p[target] (unscaled).
__global__ void ce_kernel(const float* logits, const int32_t* target, int M, int N, int B, int batch, float* g,
                          double* lpart) {
    __shared__ double red[kThreads / 32];
    const long long total = (long long)batch * N;
    const float scale = 1.f / ((float)M * (float)N * (float)batch);
    double lsum = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e % N);
        const int d = (int)(e / N);
        for (int m = 0; m < MMAX; ++m) {
            float* gr = g + ((long long)d * CH + m * QMAX) * N + n;
            if (m >= M) {
                for (int q = 0; q < QMAX; ++q) gr[(long long)q * N] = 0.f;
                continue;
            }
            const float* lr = logits + ((long long)d * CH + m * QMAX) * N + n;
            float mx = -INFINITY;
            for (int q = 0; q < B; ++q) mx = fmaxf(mx, lr[(long long)q * N]);
            float z = 0.f;
            for (int q = 0; q < B; ++q) z += expf(lr[(long long)q * N] - mx);
            const int tg = target[((long long)d * M + m) * N + n];
            lsum += (double)(logf(z) + mx - lr[(long long)tg * N]);
            const float iz = 1.f / z;
            for (int q = 0; q < QMAX; ++q) {
                float v = 0.f;
                if (q < B) v = (expf(lr[(long long)q * N] - mx) * iz - (q == tg ? 1.f : 0.f)) * scale;
                gr[(long long)q * N] = v;
            }
        }
        for (int c = MMAX * QMAX; c < CH; ++c) g[((long long)d * CH + c) * N + n] = 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        lpart[blockIdx.x] = s;
    }
}

__global__ void loss_sum_kernel(const double* lpart, int nb, double scale, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += lpart[i];
        out[0] = s * scale;
    }
}

// -------------------------------------------------------------------- Adam --
__global__ void adam_kernel(float* master, float* m, float* v, const float* grad, __half* w16, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float p = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        master[i] = p;
        w16[i] = __float2half_rn(p);
    }
}

__global__ void to_half_kernel(const float* master, __half* w16, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        w16[i] = __float2half_rn(master[i]);
}

// ------------------------------------------------------------------ argmax --
__global__ void argmax_kernel(const float* logits, int M, int N, int B, int batch, int32_t* b) {
    const long long total = (long long)batch * M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e % N);
        const int m = (int)((e / N) % M);
        const int d = (int)(e / ((long long)N * M));
        const float* lr = logits + ((long long)d * CH + m * QMAX) * N + n;
        int best = 0;
        float bv = lr[0];
        for (int q = 1; q < B; ++q) {
            const float vq = lr[(long long)q * N];
            if (vq > bv) { bv = vq; best = q; }
        }
        b[e] = best;
    }
}

}  // namespace ws

using namespace ws;

struct ws_net {
    int batch_max = 0, n_max = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    float* master = nullptr;    // [kParams]
    __half* w16 = nullptr;      // [kParams] (FP16 images; the bias slots are unused)
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* part = nullptr;      // [kSplits][64][64*5+1]
    float* act[5] = {};         // features (32 ch), three tanh layers, logits (64 ch)
    float* g[2] = {};           // dL/dz ping-pong [batch][64][N]
    double* lpart = nullptr;
    double* loss = nullptr;
    int ce_blocks = 0;
    long long t = 0;            // Adam steps taken
};

namespace {

af_status fail(ws_net* w, af_status s, const std::string& msg) {
    if (w) w->err = msg;
    return s;
}

#define WS_CK(w, call)                                                                              \
    do {                                                                                            \
        cudaError_t _e = (call);                                                                    \
        if (_e != cudaSuccess) return fail(w, AF_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(_e)); \
    } while (0)

af_status check_cfg(ws_net* w, const ws_config* c, int batch) {
    if (!c) return fail(w, AF_ERR_INVALID_ARG, "cfg is NULL");
    if (c->M < 1 || c->M > MMAX) return fail(w, AF_ERR_INVALID_ARG, "M must be in 1..4");
    if (c->B < 2 || c->B > QMAX) return fail(w, AF_ERR_INVALID_ARG, "B must be in 2..16");
    if (c->N < 1 || c->N > w->n_max) return fail(w, AF_ERR_INVALID_ARG, "N must be in 1..n_max");
    if (batch < 1 || batch > w->batch_max) return fail(w, AF_ERR_INVALID_ARG, "batch must be in 1..batch_max");
    for (int i = 0; i < 5; ++i)
        if (!isfinite(c->cond[i])) return fail(w, AF_ERR_INVALID_ARG, "cond must be finite");
    return AF_OK;
}

int grid_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

af_status run_forward(ws_net* w, const ws_config* c, int batch, const int32_t* b0) {
    const int N = c->N;
    cudaStream_t s = w->stream;
    features_kernel<<<grid_for((long long)batch * CIN * N), kThreads, 0, s>>>(
        b0, c->M, N, c->B, (float)c->cond[0], (float)c->cond[1], (float)c->cond[2], (float)c->cond[3],
        (float)c->cond[4], w->act[0], batch);
    WS_CK(w, cudaGetLastError());
    WS_CK(w, (launch_conv<CIN, FWD_TANH>(w->act[0], w->w16 + woff(0), w->master + boff(0), nullptr, w->act[1], N,
                                        batch, s)));
    WS_CK(w, (launch_conv<CH, FWD_TANH>(w->act[1], w->w16 + woff(1), w->master + boff(1), nullptr, w->act[2], N,
                                       batch, s)));
    WS_CK(w, (launch_conv<CH, FWD_TANH>(w->act[2], w->w16 + woff(2), w->master + boff(2), nullptr, w->act[3], N,
                                       batch, s)));
    WS_CK(w, (launch_conv<CH, FWD_LINEAR>(w->act[3], w->w16 + woff(3), w->master + boff(3), nullptr, w->act[4], N,
                                         batch, s)));
    return AF_OK;
}

// loss into w->loss (device), gradient into w->grad
af_status run_loss_grad(ws_net* w, const ws_config* c, int batch, const int32_t* b0, const int32_t* target) {
    af_status st = run_forward(w, c, batch, b0);
    if (st != AF_OK) return st;
    const int N = c->N;
    cudaStream_t s = w->stream;
    ce_kernel<<<w->ce_blocks, kThreads, 0, s>>>(w->act[4], target, c->M, N, c->B, batch, w->g[0], w->lpart);
    WS_CK(w, cudaGetLastError());
    loss_sum_kernel<<<1, 32, 0, s>>>(w->lpart, w->ce_blocks, 1.0 / ((double)c->M * N * batch), w->loss);
    WS_CK(w, cudaGetLastError());
    int cur = 0;
    for (int l = 3; l >= 0; --l) {
        const int ci = (l == 0) ? CIN : CH;
        dim3 grid(CH, kSplits);
        if (l == 0)
            wgrad_kernel<CIN><<<grid, CIN * KW + 32, 0, s>>>(w->g[cur], w->act[0], w->part, N, batch);
        else
            wgrad_kernel<CH><<<grid, CH * KW + 32, 0, s>>>(w->g[cur], w->act[l], w->part, N, batch);
        WS_CK(w, cudaGetLastError());
        wgrad_reduce_kernel<<<grid_for((long long)CH * (ci * KW + 1)), kThreads, 0, s>>>(
            w->part, ci, w->grad + woff(l), w->grad + boff(l));
        WS_CK(w, cudaGetLastError());
        if (l > 0) {
            // dL/dz_{l-1} = (W_l^T * dL/dz_l) (1 - a_{l}^2), a_l = input activation of layer l
            WS_CK(w, (launch_conv<CH, BWD_DATA>(w->g[cur], w->w16 + woff(l), nullptr, w->act[l], w->g[1 - cur], N,
                                               batch, s)));
            cur = 1 - cur;
        }
    }
    return AF_OK;
}

}  // namespace

extern "C" int64_t ws_param_count(void) { return kParams; }

extern "C" af_status ws_create(int32_t batch_max, int32_t n_max, void* stream, ws_net** out) {
    if (!out) return AF_ERR_INVALID_ARG;
    *out = nullptr;
    if (batch_max < 1 || n_max < 1 || (long long)batch_max * n_max > (1LL << 22)) return AF_ERR_INVALID_ARG;
    ws_net* w = new ws_net();
    w->batch_max = batch_max;
    w->n_max = n_max;
    w->stream = (cudaStream_t)stream;
    const long long BN = (long long)batch_max * n_max;
    w->ce_blocks = grid_for(BN);
    bool ok = cudaMalloc((void**)&w->master, sizeof(float) * kParams) == cudaSuccess &&
              cudaMalloc((void**)&w->w16, sizeof(__half) * kParams) == cudaSuccess &&
              cudaMalloc((void**)&w->m, sizeof(float) * kParams) == cudaSuccess &&
              cudaMalloc((void**)&w->v, sizeof(float) * kParams) == cudaSuccess &&
              cudaMalloc((void**)&w->grad, sizeof(float) * kParams) == cudaSuccess &&
              cudaMalloc((void**)&w->part, sizeof(float) * kSplits * CH * (CH * KW + 1)) == cudaSuccess &&
              cudaMalloc((void**)&w->act[0], sizeof(float) * BN * CIN) == cudaSuccess &&
              cudaMalloc((void**)&w->lpart, sizeof(double) * w->ce_blocks) == cudaSuccess &&
              cudaMalloc((void**)&w->loss, sizeof(double)) == cudaSuccess;
    for (int i = 1; ok && i < 5; ++i) ok = cudaMalloc((void**)&w->act[i], sizeof(float) * BN * CH) == cudaSuccess;
    for (int i = 0; ok && i < 2; ++i) ok = cudaMalloc((void**)&w->g[i], sizeof(float) * BN * CH) == cudaSuccess;
    if (ok)
        ok = cudaMemset(w->master, 0, sizeof(float) * kParams) == cudaSuccess &&
             cudaMemset(w->w16, 0, sizeof(__half) * kParams) == cudaSuccess &&
             cudaMemset(w->m, 0, sizeof(float) * kParams) == cudaSuccess &&
             cudaMemset(w->v, 0, sizeof(float) * kParams) == cudaSuccess;
    if (!ok) {
        ws_destroy(w);
        return AF_ERR_OOM;
    }
    *out = w;
    return AF_OK;
}

extern "C" af_status ws_destroy(ws_net* w) {
    if (!w) return AF_ERR_INVALID_ARG;
    if (w->stream) cudaStreamSynchronize(w->stream);
    void* ptrs[] = {w->master, w->w16, w->m, w->v, w->grad, w->part, w->lpart, w->loss,
                    w->act[0], w->act[1], w->act[2], w->act[3], w->act[4], w->g[0], w->g[1]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete w;
    return AF_OK;
}

extern "C" const char* ws_last_error(const ws_net* w) { return w ? w->err.c_str() : ""; }

extern "C" af_status ws_set_params(ws_net* w, const float* params_host) {
    if (!w || !params_host) return AF_ERR_INVALID_ARG;
    for (long long i = 0; i < kParams; ++i)
        if (!isfinite(params_host[i])) return fail(w, AF_ERR_INVALID_ARG, "parameters must be finite");
    WS_CK(w, cudaStreamSynchronize(w->stream));
    WS_CK(w, cudaMemcpy(w->master, params_host, sizeof(float) * kParams, cudaMemcpyHostToDevice));
    WS_CK(w, cudaMemset(w->m, 0, sizeof(float) * kParams));
    WS_CK(w, cudaMemset(w->v, 0, sizeof(float) * kParams));
    to_half_kernel<<<grid_for(kParams), kThreads, 0, w->stream>>>(w->master, w->w16, kParams);
    WS_CK(w, cudaGetLastError());
    WS_CK(w, cudaStreamSynchronize(w->stream));
    w->t = 0;
    return AF_OK;
}

extern "C" af_status ws_get_params(ws_net* w, float* params_host) {
    if (!w || !params_host) return AF_ERR_INVALID_ARG;
    WS_CK(w, cudaStreamSynchronize(w->stream));
    WS_CK(w, cudaMemcpy(params_host, w->master, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    return AF_OK;
}

extern "C" af_status ws_forward(ws_net* w, const ws_config* c, int32_t batch, const int32_t* b0_dev,
                                float* logits_dev, int32_t* b_dev) {
    if (!w) return AF_ERR_INVALID_ARG;
    af_status st = check_cfg(w, c, batch);
    if (st != AF_OK) return st;
    if (!b0_dev) return fail(w, AF_ERR_INVALID_ARG, "b0 is NULL");
    if ((st = run_forward(w, c, batch, b0_dev)) != AF_OK) return st;
    const long long n_logits = (long long)batch * CH * c->N;
    if (logits_dev)
        WS_CK(w, cudaMemcpyAsync(logits_dev, w->act[4], sizeof(float) * n_logits, cudaMemcpyDeviceToDevice, w->stream));
    if (b_dev) {
        argmax_kernel<<<grid_for((long long)batch * c->M * c->N), kThreads, 0, w->stream>>>(w->act[4], c->M, c->N, c->B,
                                                                                             batch, b_dev);
        WS_CK(w, cudaGetLastError());
    }
    return AF_OK;
}

extern "C" af_status ws_loss_grad(ws_net* w, const ws_config* c, int32_t batch, const int32_t* b0_dev,
                                  const int32_t* target_dev, double* loss_host, float* grad_host) {
    if (!w) return AF_ERR_INVALID_ARG;
    af_status st = check_cfg(w, c, batch);
    if (st != AF_OK) return st;
    if (!b0_dev || !target_dev) return fail(w, AF_ERR_INVALID_ARG, "b0 and target must not be NULL");
    if ((st = run_loss_grad(w, c, batch, b0_dev, target_dev)) != AF_OK) return st;
    WS_CK(w, cudaStreamSynchronize(w->stream));
    if (loss_host) WS_CK(w, cudaMemcpy(loss_host, w->loss, sizeof(double), cudaMemcpyDeviceToHost));
    if (grad_host) WS_CK(w, cudaMemcpy(grad_host, w->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    return AF_OK;
}

extern "C" af_status ws_train_step(ws_net* w, const ws_config* c, int32_t batch, const int32_t* b0_dev,
                                   const int32_t* target_dev, float lr, double* loss_host) {
    if (!w) return AF_ERR_INVALID_ARG;
    af_status st = check_cfg(w, c, batch);
    if (st != AF_OK) return st;
    if (!b0_dev || !target_dev) return fail(w, AF_ERR_INVALID_ARG, "b0 and target must not be NULL");
    if (!(lr > 0.f) || !isfinite(lr)) return fail(w, AF_ERR_INVALID_ARG, "lr must be finite and > 0");
    if ((st = run_loss_grad(w, c, batch, b0_dev, target_dev)) != AF_OK) return st;
    w->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - pow(0.9, (double)w->t)), c2 = (float)(1.0 - pow(0.999, (double)w->t));
    adam_kernel<<<grid_for(kParams), kThreads, 0, w->stream>>>(w->master, w->m, w->v, w->grad, w->w16, kParams, lr, b1,
                                                               b2, 1e-8f, c1, c2);
    WS_CK(w, cudaGetLastError());
    if (loss_host) {
        WS_CK(w, cudaStreamSynchronize(w->stream));
        WS_CK(w, cudaMemcpy(loss_host, w->loss, sizeof(double), cudaMemcpyDeviceToHost));
    }
    return AF_OK;
}
