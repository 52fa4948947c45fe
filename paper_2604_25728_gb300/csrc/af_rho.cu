// af_rho.cu -- trainable quantization thresholds (Section III-C: the rho_i of
// Eq. 24 are trained jointly with the transmit parameters in Step B of
// Algorithm 1, and kept an ordered set).
//
//   rho_grad_kernel (one thread per element, the K thresholds staged in
//   shared memory): dL/drho_i += dL/dy_e * (-a c (1 - tanh^2(c (z_e - rho_i))))
//   over the thresholds within the tanh window of z_e.  Terms are summed as
//   64-bit fixed point (scale 2^40), first per CTA in shared memory, then
//   into a global accumulator: integer sums do not depend on the order of
//   the atomics, so the gradient is reproducible.
//   rho_kernel (one CTA): reads and clears the accumulator, then Adam on rho
//   (the Step-B step counter, as for the logits) and the projection onto
//   0 <= rho_0 <= ... <= rho_{K-1} <= 1 (a parallel test, and only when it
//   fails the pool-adjacent-violators pass, by one thread: its cost grows
//   with K, and small steps rarely break the order).
// dL/dy_e and z_e come from the finish kernel of the same evaluation, which
// writes them before it updates the logits; the next waveform is formed
// afterwards by wave_from_logits with the updated thresholds.
#include <math.h>

#include "af_device.cuh"
#include "af_kernels.h"
#include "af_step.cuh"

namespace af {

constexpr int kRhoThreads = 1024;
constexpr float kFixScaleF = 1099511627776.0f;  // 2^40, exact in FP32
constexpr float kFixInvF = 1.0f / 1099511627776.0f;  // 2^-40, exact

int rho_smem_bytes(int K) { return K * (int)(sizeof(float) + sizeof(long long) + sizeof(int)); }
static int rho_grad_smem_bytes(int K) { return K * (int)(sizeof(float) + sizeof(long long)); }
constexpr int kRhoGradThreads = 256;

__global__ void __launch_bounds__(kRhoGradThreads) rho_grad_kernel(const RhoArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = a.q.K;
    long long* acc = reinterpret_cast<long long*>(smem_raw);          // [K]
    float* rs = reinterpret_cast<float*>(acc + K);                    // [K]
    const int tid = threadIdx.x;
    pdl_wait();
    for (int i = tid; i < K; i += kRhoGradThreads) { rs[i] = a.rho[i]; acc[i] = 0; }
    QuantArgs q = a.q;
    q.rho = rs;
    q.uniform = 0;
    __syncthreads();
    const int e = blockIdx.x * kRhoGradThreads + tid;
    if (e < a.n) {
        const float ac = q.a * q.c;
        const float z = a.z[e], gy = a.gy[e];
        const int i0 = count_lt(q, z - q.win), i1 = count_le(q, z + q.win);
        for (int i = i0; i < i1; ++i) {
            const float t = tanhf(q.c * (z - rs[i]));
            const float g = -gy * ac * (1.f - t * t);
            // scaling by 2^40 is exact in FP32; the conversion rounds once (no FP64 in the loop)
            atomicAdd(reinterpret_cast<unsigned long long*>(acc + i),
                      (unsigned long long)__float2ll_rn(g * kFixScaleF));
        }
    }
    __syncthreads();
    for (int i = tid; i < K; i += kRhoGradThreads)
        if (acc[i] != 0) atomicAdd(reinterpret_cast<unsigned long long*>(a.acc + i), (unsigned long long)acc[i]);
}

__global__ void __launch_bounds__(kRhoThreads) rho_kernel(const RhoArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = a.q.K;
    float* rs = reinterpret_cast<float*>(smem_raw);                   // [K] thresholds
    int* cnt = reinterpret_cast<int*>(rs + K);                        // [K] pool sizes (projection)
    float* val = reinterpret_cast<float*>(cnt + K);                   // [K] pool means
    __shared__ float s_adam[2];
    const int tid = threadIdx.x;

    pdl_wait();
    for (int i = tid; i < K; i += kRhoThreads) rs[i] = a.rho[i];
    if (a.mode == RHO_GRAD || a.mode == RHO_STEP) {
        if (a.mode == RHO_GRAD) {
            for (int i = tid; i < K; i += kRhoThreads) {
                a.grad_out[i] = (float)a.acc[i] * kFixInvF;
                a.acc[i] = 0;
            }
            return;
        }
        if (tid == 0) {
            const long long t = a.ctr[2] + (a.ctr[0] - 1) * a.n_x + a.inner + 1;
            s_adam[0] = -expm1f((float)t * log1pf(a.b1 - 1.f));
            s_adam[1] = -expm1f((float)t * log1pf(a.b2 - 1.f));
        }
        __syncthreads();
        const float c1 = s_adam[0], c2 = s_adam[1];
        for (int i = tid; i < K; i += kRhoThreads) {
            const float g = (float)a.acc[i] * kFixInvF;
            a.acc[i] = 0;
            const float m = a.b1 * a.m_rho[i] + (1.f - a.b1) * g;
            const float v = a.b2 * a.v_rho[i] + (1.f - a.b2) * g * g;
            a.m_rho[i] = m;
            a.v_rho[i] = v;
            rs[i] -= a.lr * (m / c1) / (sqrtf(v / c2) + a.adam_eps);
        }
    }
    __syncthreads();

    // ---- projection onto the ordered set inside [0, 1] ----
    bool bad = false;
    for (int i = tid; i < K; i += kRhoThreads)
        bad |= !(rs[i] >= 0.f && rs[i] <= 1.f) || (i + 1 < K && rs[i + 1] < rs[i]);
    if (__syncthreads_or(bad)) {
        if (tid == 0) {
            int nb = 0;
            for (int i = 0; i < K; ++i) {
                val[nb] = rs[i];
                cnt[nb] = 1;
                ++nb;
                while (nb > 1 && val[nb - 2] > val[nb - 1]) {
                    const int c = cnt[nb - 2] + cnt[nb - 1];
                    val[nb - 2] = (val[nb - 2] * (float)cnt[nb - 2] + val[nb - 1] * (float)cnt[nb - 1]) / (float)c;
                    cnt[nb - 2] = c;
                    --nb;
                }
            }
            int i = 0;
            for (int b = 0; b < nb; ++b) {
                const float v = fminf(fmaxf(val[b], 0.f), 1.f);
                for (int r = 0; r < cnt[b]; ++r) rs[i++] = v;
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < K; i += kRhoThreads) a.rho[i] = rs[i];
}

cudaError_t rho_prepare(int K) {
    cudaError_t e = set_smem_once(reinterpret_cast<const void*>(rho_kernel), rho_smem_bytes(K));
    if (e != cudaSuccess) return e;
    return set_smem_once(reinterpret_cast<const void*>(rho_grad_kernel), rho_grad_smem_bytes(K));
}

// RHO_GRAD and RHO_STEP: the per-element kernel accumulates, then the single
// CTA reads the sum; RHO_PROJECT: the single CTA alone.
cudaError_t launch_rho(const RhoArgs& a, cudaStream_t s) {
    if (a.mode == RHO_GRAD || a.mode == RHO_STEP) {
        cudaError_t e = launch_ex(rho_grad_kernel, dim3((a.n + kRhoGradThreads - 1) / kRhoGradThreads),
                                  dim3(kRhoGradThreads), (size_t)rho_grad_smem_bytes(a.q.K), s, a.pdl != 0, a);
        if (e != cudaSuccess) return e;
    }
    return launch_ex(rho_kernel, dim3(1), dim3(kRhoThreads), (size_t)rho_smem_bytes(a.q.K), s, a.pdl != 0, a);
}

}  // namespace af
