// af_step.cu -- transmit chain, loss assembly, sparse adjoint, Adam and the
// energy projection: everything of one evaluation that is O(M N).
//
//  * wave kernels: z = sigmoid(u); soft waveform x = e^{j 2 pi Q_A(z)} with
//    dQ_A/dz (Eq. 24, copies K = B r_n); hard waveform from q = #{rho_i <= z}
//    (Eq. 43 in the c -> infinity reading).
//  * fin kernel (one CTA per waveform row m): merges the per-CTA sidelobe
//    partials of the forward pass into WAPSL/WCPSL (Eqs. 8-9), L_WPSL
//    (Eq. 37), p_m (Eq. 38), L_SNRL (Eq. 41) and L (Eq. 42); then forms row m
//    of the gradient: the exact max is differentiated at its winning cell
//    (k*, nu*) of pair (m*, l*):
//        grad x_m*(n)  += g h_l*(n+k*) e^{-j 2 pi nu* n}
//        grad h_l*(p)  += conj(g) x_m*(p-k*) e^{+j 2 pi nu* (p-k*)}
//    with g = eps w chi*/|chi*|, plus the SNRL term at (m, m, 0, 0), plus (in
//    the p-norm variant) the dense partial gradients of the adjoint kernel.
//    The chain to the logits is dL/du = 2 pi Im(conj(x) grad x) Q_A'(z) z(1-z).
//    In the optimiser modes the same CTA applies Adam (and, for the filters,
//    the projection of Eq. 32 with an FP64 norm) and prepares the waveform of
//    the next evaluation.
#include <math.h>

#include "af_common.cuh"
#include "af_kernels.h"
#include "af_step.cuh"
#include "af_device.cuh"

namespace af {

constexpr int kFinThreads = 256;

// ------------------------------------------------------------ wave kernels --
// A table of thresholds that is not the uniform set (user-set or trained) is
// staged in shared memory when it fits, so that the binary searches of the
// quantizers read shared rather than global memory.
constexpr int kStageK = 8192;

__global__ void wave_from_logits_kernel(const float* __restrict__ u, int n, QuantArgs q, int hard,
                                        float2* __restrict__ x, float* __restrict__ dydz,
                                        int32_t* __restrict__ qout) {
    extern __shared__ float rho_s[];
    if (!q.uniform && q.K <= kStageK) {
        for (int k = threadIdx.x; k < q.K; k += blockDim.x) rho_s[k] = q.rho[k];
        __syncthreads();
        q.rho = rho_s;
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float z = sigmoidf_(u[i]);
    if (hard) {
        const int qq = hard_q(q, z);
        if (x) x[i] = q.level[qq % q.B];
        if (qout) qout[i] = qq;
    } else {
        float2 xv;
        float d;
        soft_q(q, z, nullptr, &d, &xv);
        if (x) x[i] = xv;
        if (dydz) dydz[i] = d;
    }
}

__global__ void quantize_z_kernel(const float* __restrict__ z, long long n, QuantArgs q,
                                  int32_t* __restrict__ qout, float2* __restrict__ x) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int qq = hard_q(q, z[i]);
    if (qout) qout[i] = qq;
    if (x) x[i] = q.level[qq % q.B];
}

__global__ void soft_quantize_z_kernel(const float* __restrict__ z, long long n, QuantArgs q,
                                       float* __restrict__ y, float* __restrict__ dydz,
                                       float2* __restrict__ x) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float yy, dd;
    float2 xv;
    soft_q(q, z[i], &yy, &dd, &xv);
    if (y) y[i] = yy;
    if (dydz) dydz[i] = dd;
    if (x) x[i] = xv;
}

// FP64 hard waveform and FP64 copy of the filters for the acceptance pass
// (h == nullptr: matched filters, h64 = x64).
__global__ void wave_hard_f64_kernel(const float* __restrict__ u, const float2* __restrict__ h, int n,
                                     QuantArgs q, const double2* __restrict__ level64,
                                     double2* __restrict__ x64, double2* __restrict__ h64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int qq = hard_q(q, sigmoidf_(u[i]));
    const double2 xv = level64[qq % q.B];
    x64[i] = xv;
    if (h == nullptr) {
        h64[i] = xv;
    } else {
        const float2 hv = h[i];
        h64[i] = make_double2((double)hv.x, (double)hv.y);
    }
}

// -------------------------------------------------------------- projection --
__global__ void __launch_bounds__(kFinThreads) project_kernel(float2* h, int N) {
    __shared__ double shd[kFinThreads / 32];
    const int m = blockIdx.x;
    double e2 = 0.0;
    for (int n = threadIdx.x; n < N; n += kFinThreads) {
        const float2 v = h[(size_t)m * N + n];
        e2 += (double)v.x * v.x + (double)v.y * v.y;
    }
    e2 = block_sum_d(e2, shd);
    if (!(e2 > 0.0)) return;
    const float sc = (float)sqrt((double)N / e2);
    for (int n = threadIdx.x; n < N; n += kFinThreads) {
        const float2 v = h[(size_t)m * N + n];
        h[(size_t)m * N + n] = make_float2(v.x * sc, v.y * sc);
    }
}

// ------------------------------------------------------------------ init ----
__global__ void init_kernel(const int32_t* __restrict__ b, const float2* __restrict__ noise, int n,
                            int B, int r_n, QuantArgs q, float* __restrict__ u, float2* __restrict__ h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int bb = b[i];
    const double K = (double)B * r_n;
    const double z0 = ((double)(r_n / 2) * B + bb) / K;
    u[i] = (float)log(z0 / (1.0 - z0));
    float2 hv = q.level[((bb % B) + B) % B];
    if (noise) hv = cadd(hv, noise[i]);
    h[i] = hv;
}

// ----------------------------------------------------------- acceptance -----
__global__ void __launch_bounds__(kFinThreads) acceptance_kernel(const AccArgs a) {
    __shared__ double shd[kFinThreads / 32];
    __shared__ double sk[2][kFinThreads / 32];
    const int tid = threadIdx.x;
    double kb[2] = {-1.0, -1.0};
    for (int b = tid; b < a.nblk; b += kFinThreads) {
        const int pair = b / a.ctas_per_pair;
        const int cls = (pair / a.M == pair % a.M) ? 0 : 1;
        kb[cls] = fmax(kb[cls], a.pkey[b]);
    }
    for (int c = 0; c < 2; ++c) {
        for (int o = 16; o > 0; o >>= 1) kb[c] = fmax(kb[c], __shfl_xor_sync(0xffffffffu, kb[c], o));
        if ((tid & 31) == 0) sk[c][tid >> 5] = kb[c];
    }
    __syncthreads();
    if (tid == 0) {
        for (int c = 0; c < 2; ++c) {
            double k = sk[c][0];
            for (int w = 1; w < kFinThreads / 32; ++w) k = fmax(k, sk[c][w]);
            a.out[c] = (k > 0.0) ? 20.0 * log10(sqrt(k) / a.N) : -INFINITY;
        }
        a.out[2] = fmax(a.out[0], a.out[1]);
    }
    // SNRL (Eq. 10) for every m, FP64
    double smax = -INFINITY;
    for (int m = 0; m < a.M; ++m) {
        double ex = 0.0, eh = 0.0;
        for (int n = tid; n < a.N; n += kFinThreads) {
            const double2 xv = a.x[(size_t)m * a.N + n], hv = a.h[(size_t)m * a.N + n];
            ex += xv.x * xv.x + xv.y * xv.y;
            eh += hv.x * hv.x + hv.y * hv.y;
        }
        ex = block_sum_d(ex, shd);
        eh = block_sum_d(eh, shd);
        const double2 c = a.cdiag[m];
        const double s = 10.0 * log10(ex * eh / (c.x * c.x + c.y * c.y));
        if (tid == 0) a.out[4 + m] = s;
        smax = fmax(smax, s);
    }
    if (tid == 0) a.out[3] = smax;
}

// ------------------------------------------------------------ launchers -----
cudaError_t launch_wave_from_logits(const float* u, int n, const QuantArgs& q, int hard, float2* x,
                                    float* dydz, int32_t* qout, cudaStream_t s) {
    const size_t smem = (!q.uniform && q.K <= kStageK) ? sizeof(float) * q.K : 0;
    wave_from_logits_kernel<<<(n + 255) / 256, 256, smem, s>>>(u, n, q, hard, x, dydz, qout);
    return cudaGetLastError();
}
cudaError_t launch_quantize_z(const float* z, long long n, const QuantArgs& q, int32_t* qout, float2* x,
                              cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    quantize_z_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(z, n, q, qout, x);
    return cudaGetLastError();
}
cudaError_t launch_soft_quantize_z(const float* z, long long n, const QuantArgs& q, float* y, float* dydz,
                                   float2* x, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    soft_quantize_z_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(z, n, q, y, dydz, x);
    return cudaGetLastError();
}
cudaError_t launch_wave_hard_f64(const float* u, const float2* h, int n, const QuantArgs& q,
                                 const double2* level64, double2* x64, double2* h64, cudaStream_t s) {
    wave_hard_f64_kernel<<<(n + 255) / 256, 256, 0, s>>>(u, h, n, q, level64, x64, h64);
    return cudaGetLastError();
}
cudaError_t launch_project(float2* h, int M, int N, cudaStream_t s) {
    project_kernel<<<M, kFinThreads, 0, s>>>(h, N);
    return cudaGetLastError();
}
cudaError_t launch_init(const int32_t* b, const float2* noise, int n, int B, int r_n, const QuantArgs& q,
                        float* u, float2* h, cudaStream_t s) {
    init_kernel<<<(n + 255) / 256, 256, 0, s>>>(b, noise, n, B, r_n, q, u, h);
    return cudaGetLastError();
}
cudaError_t launch_acceptance(const AccArgs& a, cudaStream_t s) {
    acceptance_kernel<<<1, kFinThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace af

namespace af {

__global__ void set_counters_kernel(long long* ctr, long long a0, long long a1, long long a2, long long a3) {
    ctr[0] = a0; ctr[1] = a1; ctr[2] = a2; ctr[3] = a3;
}
__global__ void copy_f64_kernel(double* dst, const double* src, int n) {
    const int i = threadIdx.x;
    if (i < n) dst[i] = src[i];
}
cudaError_t launch_set_counters(long long* ctr, long long a0, long long a1, long long a2, long long a3,
                                cudaStream_t s) {
    set_counters_kernel<<<1, 1, 0, s>>>(ctr, a0, a1, a2, a3);
    return cudaGetLastError();
}
cudaError_t launch_copy_f64(double* dst, const double* src, int n, cudaStream_t s) {
    copy_f64_kernel<<<1, 32, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

}  // namespace af
