// af_rn.cu -- the transmit-side ResNet generator z = f_theta(y0) (Eq. 17; the
// architecture of Section IV: 5 residual blocks of width 128, tanh hidden and
// residual layers, sigmoid output):
//     h_0 = tanh(W_in y0 + b_in)
//     r_k = tanh(W1_k h_{k-1} + b1_k),  h_k = tanh(h_{k-1} + W2_k r_k + b2_k)
//     u   = W_out h_5 + b_out,          z = sigmoid(u)
// with one Adam step on every parameter per transmit evaluation, given
// du = dL/du from the finish kernel.
//
// The input is one fixed vector, so every layer is a matrix-vector product:
// bandwidth-bound on the weights (2 H P of the 2 H P + 10 H^2 parameters sit in
// the first and last layers), not a tensor-core contraction.  Five kernels per
// step, each reading its weights once:
//   out_bwd   (P/64 CTAs)  Adam on W_out, b_out; per-CTA partials of W_out^T du
//   blocks_bwd (cluster)   the partials summed, the 5 blocks backward with
//                          Adam, da = dL/d(W_in y0 + b_in)
//   in_step   (P/64 CTAs)  Adam on W_in (and b_in in CTA 0); per-CTA partials
//                          of the new W_in y0
//   blocks_fwd (cluster)   h_0 .. h_5 with the new weights
//   out_fwd   (P/64 CTAs)  u = W_out h_5 + b_out and the next waveform
// The cluster kernels give each of their kCS CTAs 128/kCS rows of every
// block matrix and exchange the 128-vectors between layers through
// distributed shared memory; every cross-CTA sum is taken in a fixed order.
#include <math.h>
#include <stdio.h>

#include <string>

#include "../../include/resnet.h"
#include "af_device.cuh"
#include "af_kernels.h"
#include "af_step.cuh"
#include "af_tc.cuh"

namespace af {
namespace {

constexpr int kH = 128;            // hidden width
constexpr int kBlocks = 5;
constexpr int kCS = 8;             // CTAs per cluster in the block kernels
constexpr int kRW = kH / kCS;      // block-matrix rows per cluster CTA
constexpr int kT = 256;            // threads per CTA
constexpr int kRB = 64;            // output rows (out_*) or input columns (in_step) per CTA

struct RnOffsets {
    long long w_in, b_in, blk, w_out, b_out, total;
    __host__ __device__ long long w1(int k) const { return blk + (long long)k * (2 * kH * kH + 2 * kH); }
    __host__ __device__ long long b1(int k) const { return w1(k) + kH * kH; }
    __host__ __device__ long long w2(int k) const { return b1(k) + kH; }
    __host__ __device__ long long b2(int k) const { return w2(k) + kH * kH; }
};

RnOffsets offsets(int P) {
    RnOffsets o;
    o.w_in = 0;
    o.b_in = (long long)kH * P;
    o.blk = o.b_in + kH;
    o.w_out = o.blk + (long long)kBlocks * (2 * kH * kH + 2 * kH);
    o.b_out = o.w_out + (long long)P * kH;
    o.total = o.b_out + P;
    return o;
}

struct RnArgs {
    int P;
    RnOffsets o;
    float* th;                 // parameters, the oracle's flat order
    float* m;                  // Adam moments
    float* v;
    const float* y0;           // [P]
    const float* du;           // [P] dL/du
    float* part;               // [nPart][kH] per-CTA partial vectors
    int n_part;
    float* hs;                 // [kBlocks + 1][kH] h_0 .. h_5
    float* rs;                 // [kBlocks][kH] r_1 .. r_5
    float* da;                 // [kH]
    float* u;                  // [P] output (pre-sigmoid)
    int adam;                  // 0: forward only (in_step computes the partials, no update)
    float lr, b1, b2, eps;
    float c1, c2;              // bias corrections when ctr is null
    const long long* ctr;      // step counters: t = ctr[2] + (ctr[0] - 1) n_x + inner + 1
    int inner, n_x;
    QuantArgs q;               // next waveform
    int next_wave;
    float2* x_next;
    float* dydz_next;
    int pdl;
};

__device__ __forceinline__ void adam_consts(const RnArgs& a, float& c1, float& c2) {
    if (a.ctr == nullptr) { c1 = a.c1; c2 = a.c2; return; }
    const long long t = a.ctr[2] + (a.ctr[0] - 1) * a.n_x + a.inner + 1;
    c1 = -expm1f((float)t * log1pf(a.b1 - 1.f));
    c2 = -expm1f((float)t * log1pf(a.b2 - 1.f));
}

__device__ __forceinline__ float adam1(float& w, float& m, float& v, float g, const RnArgs& a, float c1, float c2) {
    const float w_old = w;
    m = a.b1 * m + (1.f - a.b1) * g;
    v = a.b2 * v + (1.f - a.b2) * g * g;
    w -= a.lr * (m / c1) / (sqrtf(v / c2) + a.eps);
    return w_old;
}

__device__ __forceinline__ float warp_sum_f(float x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ---------------------------------------------------------------- out_bwd --
// CTA b: rows e in [b kRB, (b+1) kRB); warp w takes rows e = base + w + 8 i;
// lane l holds columns 4l .. 4l+3.
__global__ void __launch_bounds__(kT) rn_out_bwd(const RnArgs a) {
    __shared__ float h5[kH];
    __shared__ float pw[kT / 32][kH];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_wait();
    if (tid < kH) h5[tid] = a.hs[kBlocks * kH + tid];
    float c1, c2;
    adam_consts(a, c1, c2);
    __syncthreads();
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int base = blockIdx.x * kRB;
    for (int r = warp; r < kRB; r += kT / 32) {
        const int e = base + r;
        if (e >= a.P) break;
        const float d = a.du[e];
        const long long off = a.o.w_out + (long long)e * kH + 4 * lane;
        float4 w = *reinterpret_cast<const float4*>(a.th + off);
        float4 m = *reinterpret_cast<const float4*>(a.m + off);
        float4 v = *reinterpret_cast<const float4*>(a.v + off);
        acc[0] += w.x * d; acc[1] += w.y * d; acc[2] += w.z * d; acc[3] += w.w * d;
        adam1(w.x, m.x, v.x, d * h5[4 * lane], a, c1, c2);
        adam1(w.y, m.y, v.y, d * h5[4 * lane + 1], a, c1, c2);
        adam1(w.z, m.z, v.z, d * h5[4 * lane + 2], a, c1, c2);
        adam1(w.w, m.w, v.w, d * h5[4 * lane + 3], a, c1, c2);
        *reinterpret_cast<float4*>(a.th + off) = w;
        *reinterpret_cast<float4*>(a.m + off) = m;
        *reinterpret_cast<float4*>(a.v + off) = v;
        if (lane == 0) {
            const long long ob = a.o.b_out + e;
            adam1(a.th[ob], a.m[ob], a.v[ob], d, a, c1, c2);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) pw[warp][4 * lane + q] = acc[q];
    __syncthreads();
    if (tid < kH) {
        float s = 0.f;
        for (int w = 0; w < kT / 32; ++w) s += pw[w][tid];
        a.part[(size_t)blockIdx.x * kH + tid] = s;
    }
}

// Sum of the 128-vector partials of a cluster, in rank order, into dst (all CTAs).
__device__ __forceinline__ void cluster_allsum(const float* mine, float* dst, int tid) {
    tc::cluster_sync();
    if (tid < kH) {
        const uint32_t local = tc::smem_u32(mine + tid);
        float s = 0.f;
        for (int r = 0; r < kCS; ++r) {
            uint32_t remote;
            float x;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
            asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(x) : "r"(remote) : "memory");
            s += x;
        }
        dst[tid] = s;
    }
    tc::cluster_sync();
}

// Gather the kRW-value slices of a cluster into dst[kH] (all CTAs).
__device__ __forceinline__ void cluster_gather(const float* mine, float* dst, int tid) {
    tc::cluster_sync();
    if (tid < kH) {
        const int r = tid / kRW, i = tid % kRW;
        const uint32_t local = tc::smem_u32(mine + i);
        uint32_t remote;
        float x;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
        asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(x) : "r"(remote) : "memory");
        dst[tid] = x;
    }
    tc::cluster_sync();
}

// Per-warp partial of W^T d over this CTA's rows of an H x H matrix with Adam
// on those rows (g = d_i in_j), written to pw[warp][*]; rows i0 + warp, i0 + warp + 8.
__device__ __forceinline__ void block_layer_bwd(const RnArgs& a, long long w_off, long long b_off, const float* d,
                                                const float* in, int i0, float (*pw)[kH], int lane, int warp,
                                                float c1, float c2) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int r = warp; r < kRW; r += kT / 32) {
        const int i = i0 + r;
        const float di = d[i];
        const long long off = w_off + (long long)i * kH + 4 * lane;
        float4 w = *reinterpret_cast<const float4*>(a.th + off);
        float4 m = *reinterpret_cast<const float4*>(a.m + off);
        float4 v = *reinterpret_cast<const float4*>(a.v + off);
        acc[0] += w.x * di; acc[1] += w.y * di; acc[2] += w.z * di; acc[3] += w.w * di;
        adam1(w.x, m.x, v.x, di * in[4 * lane], a, c1, c2);
        adam1(w.y, m.y, v.y, di * in[4 * lane + 1], a, c1, c2);
        adam1(w.z, m.z, v.z, di * in[4 * lane + 2], a, c1, c2);
        adam1(w.w, m.w, v.w, di * in[4 * lane + 3], a, c1, c2);
        *reinterpret_cast<float4*>(a.th + off) = w;
        *reinterpret_cast<float4*>(a.m + off) = m;
        *reinterpret_cast<float4*>(a.v + off) = v;
        if (lane == 0) adam1(a.th[b_off + i], a.m[b_off + i], a.v[b_off + i], di, a, c1, c2);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) pw[warp][4 * lane + q] = acc[q];
}

// ------------------------------------------------------------- blocks_bwd --
__global__ void __launch_bounds__(kT) rn_blocks_bwd(const RnArgs a) {
    __shared__ float dh[kH], ds[kH], dq[kH], hk[kH], hp[kH], rk[kH];
    __shared__ float pw[kT / 32][kH];
    __shared__ float mine[kH];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = tc::cluster_ctarank() * kRW;
    pdl_wait();
    float c1, c2;
    adam_consts(a, c1, c2);
    if (tid < kH) {                              // dL/dh_5 = W_out^T du (fixed order over CTAs)
        float s = 0.f;
        for (int b = 0; b < a.n_part; ++b) s += a.part[(size_t)b * kH + tid];
        dh[tid] = s;
    }
    __syncthreads();
    for (int k = kBlocks - 1; k >= 0; --k) {
        if (tid < kH) {
            hk[tid] = a.hs[(k + 1) * kH + tid];
            hp[tid] = a.hs[k * kH + tid];
            rk[tid] = a.rs[k * kH + tid];
        }
        __syncthreads();
        if (tid < kH) ds[tid] = dh[tid] * (1.f - hk[tid] * hk[tid]);
        __syncthreads();
        block_layer_bwd(a, a.o.w2(k), a.o.b2(k), ds, rk, i0, pw, lane, warp, c1, c2);
        __syncthreads();
        if (tid < kH) {
            float s = 0.f;
            for (int w = 0; w < kT / 32; ++w) s += pw[w][tid];
            mine[tid] = s;
        }
        cluster_allsum(mine, dq, tid);            // dq <- W2^T ds
        if (tid < kH) dq[tid] *= (1.f - rk[tid] * rk[tid]);
        __syncthreads();
        block_layer_bwd(a, a.o.w1(k), a.o.b1(k), dq, hp, i0, pw, lane, warp, c1, c2);
        __syncthreads();
        if (tid < kH) {
            float s = 0.f;
            for (int w = 0; w < kT / 32; ++w) s += pw[w][tid];
            mine[tid] = s;
        }
        cluster_allsum(mine, dh, tid);            // dh <- W1^T dq
        if (tid < kH) dh[tid] += ds[tid];         // + the skip path
        __syncthreads();
    }
    if (tc::cluster_ctarank() == 0 && tid < kH) {
        const float h0 = a.hs[tid];
        a.da[tid] = dh[tid] * (1.f - h0 * h0);
    }
}

// ---------------------------------------------------------------- in_step --
// CTA b: input columns j in [b kRB, (b+1) kRB) of every row; warp w takes
// rows w, w + 8, ...; lane l holds columns 2l, 2l+1.  With adam = 1 the rows
// are updated first (g = da_i y0_j); the partial of W_in y0 uses the result.
__global__ void __launch_bounds__(kT) rn_in_step(const RnArgs a) {
    __shared__ float das[kH];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_wait();
    float c1 = 1.f, c2 = 1.f;
    if (a.adam) {
        adam_consts(a, c1, c2);
        if (tid < kH) das[tid] = a.da[tid];
    }
    __syncthreads();
    const int j = blockIdx.x * kRB + 2 * lane;
    const float y_a = (j < a.P) ? a.y0[j] : 0.f, y_b = (j + 1 < a.P) ? a.y0[j + 1] : 0.f;
    for (int i = warp; i < kH; i += kT / 32) {
        const long long off = a.o.w_in + (long long)i * a.P + j;
        float wa = 0.f, wb = 0.f;
        if (j < a.P) {
            wa = a.th[off];
            if (a.adam) {
                float m = a.m[off], v = a.v[off];
                adam1(wa, m, v, das[i] * y_a, a, c1, c2);
                a.th[off] = wa; a.m[off] = m; a.v[off] = v;
            }
        }
        if (j + 1 < a.P) {
            wb = a.th[off + 1];
            if (a.adam) {
                float m = a.m[off + 1], v = a.v[off + 1];
                adam1(wb, m, v, das[i] * y_b, a, c1, c2);
                a.th[off + 1] = wb; a.m[off + 1] = m; a.v[off + 1] = v;
            }
        }
        const float s = warp_sum_f(wa * y_a + wb * y_b);
        if (lane == 0) a.part[(size_t)blockIdx.x * kH + i] = s;
    }
    if (a.adam && blockIdx.x == 0 && tid < kH) {
        const long long ob = a.o.b_in + tid;
        adam1(a.th[ob], a.m[ob], a.v[ob], das[tid], a, c1, c2);
    }
}

// Rows i0 .. i0 + kRW - 1 of W x + b for an H x H matrix: warp w computes rows
// i0 + w and i0 + w + 8 into out[].
__device__ __forceinline__ void block_layer_fwd(const RnArgs& a, long long w_off, long long b_off, const float* x,
                                                int i0, float* out, int lane, int warp) {
    for (int r = warp; r < kRW; r += kT / 32) {
        const int i = i0 + r;
        const float4 w = *reinterpret_cast<const float4*>(a.th + w_off + (long long)i * kH + 4 * lane);
        float s = w.x * x[4 * lane] + w.y * x[4 * lane + 1] + w.z * x[4 * lane + 2] + w.w * x[4 * lane + 3];
        s = warp_sum_f(s);
        if (lane == 0) out[r] = s + a.th[b_off + i];
    }
}

// ------------------------------------------------------------- blocks_fwd --
__global__ void __launch_bounds__(kT) rn_blocks_fwd(const RnArgs a) {
    __shared__ float h[kH], r[kH];
    __shared__ float mine[kRW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = tc::cluster_ctarank();
    const int i0 = rank * kRW;
    pdl_wait();
    if (tid < kH) {                              // h_0 = tanh(W_in y0 + b_in), fixed order over CTAs
        float s = a.th[a.o.b_in + tid];
        for (int b = 0; b < a.n_part; ++b) s += a.part[(size_t)b * kH + tid];
        h[tid] = tanhf(s);
        if (rank == 0) a.hs[tid] = h[tid];
    }
    __syncthreads();
    for (int k = 0; k < kBlocks; ++k) {
        block_layer_fwd(a, a.o.w1(k), a.o.b1(k), h, i0, mine, lane, warp);
        __syncthreads();
        if (tid < kRW) mine[tid] = tanhf(mine[tid]);
        cluster_gather(mine, r, tid);             // r_k
        if (rank == 0 && tid < kH) a.rs[k * kH + tid] = r[tid];
        block_layer_fwd(a, a.o.w2(k), a.o.b2(k), r, i0, mine, lane, warp);
        __syncthreads();
        if (tid < kRW) mine[tid] = tanhf(h[i0 + tid] + mine[tid]);
        cluster_gather(mine, h, tid);             // h_k
        if (rank == 0 && tid < kH) a.hs[(k + 1) * kH + tid] = h[tid];
    }
}

// ---------------------------------------------------------------- out_fwd --
__global__ void __launch_bounds__(kT) rn_out_fwd(const RnArgs a) {
    __shared__ float h5[kH];
    __shared__ float us[kRB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_wait();
    pdl_trigger();
    if (tid < kH) h5[tid] = a.hs[kBlocks * kH + tid];
    __syncthreads();
    const int base = blockIdx.x * kRB;
    for (int r = warp; r < kRB; r += kT / 32) {
        const int e = base + r;
        if (e >= a.P) break;
        const float4 w = *reinterpret_cast<const float4*>(a.th + a.o.w_out + (long long)e * kH + 4 * lane);
        float s = w.x * h5[4 * lane] + w.y * h5[4 * lane + 1] + w.z * h5[4 * lane + 2] + w.w * h5[4 * lane + 3];
        s = warp_sum_f(s);
        if (lane == 0) us[r] = s + a.th[a.o.b_out + e];
    }
    __syncthreads();
    if (tid < kRB && base + tid < a.P) {
        const int e = base + tid;
        const float u = us[tid];
        a.u[e] = u;
        if (a.next_wave != NEXT_NONE) {
            const float z = sigmoidf_(u);
            if (a.next_wave == NEXT_HARD) {
                a.x_next[e] = a.q.level[hard_q(a.q, z) % a.q.B];
            } else {
                float2 xv;
                float d;
                soft_q(a.q, z, nullptr, &d, &xv);
                a.x_next[e] = xv;
                a.dydz_next[e] = d;
            }
        }
    }
}

cudaError_t launch_cluster(void (*kern)(RnArgs), const RnArgs& a, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCS);
    cfg.blockDim = dim3(kT);
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kCS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    int na = 1;
    if (a.pdl) {
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        na = 2;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace
}  // namespace af

using namespace af;

struct rn_net {
    int P = 0;
    RnOffsets o{};
    float* th = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* part = nullptr;
    int n_part = 0;
    float* hs = nullptr;
    float* rs = nullptr;
    float* da = nullptr;
    float* u = nullptr;        // output of rn_forward when the caller passes none
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {
thread_local std::string g_rn_error;   // failures with no network to hold the message, one per thread
#define RN_FAIL(n, code, ...)                                         \
    do {                                                              \
        char b_[256];                                                 \
        snprintf(b_, sizeof b_, __VA_ARGS__);                         \
        if (n) (n)->err = b_; else g_rn_error = b_;                   \
        return code;                                                  \
    } while (0)
#define RN_CK(n, x)                                                                  \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) RN_FAIL(n, AF_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)

RnArgs base_args(const rn_net* n) {
    RnArgs a{};
    a.P = n->P;
    a.o = n->o;
    a.th = n->th; a.m = n->m; a.v = n->v;
    a.part = n->part; a.n_part = n->n_part;
    a.hs = n->hs; a.rs = n->rs; a.da = n->da;
    a.b1 = 0.9f; a.b2 = 0.999f; a.eps = 1e-8f;
    return a;
}
}  // namespace

namespace af {
namespace {
// One training step (when adam) and the forward pass, on stream s.
cudaError_t rn_enqueue(rn_net* n, const RnArgs& in, cudaStream_t s) {
    RnArgs a = in;
    const unsigned g = (unsigned)((n->P + kRB - 1) / kRB);
    cudaError_t e = cudaSuccess;
    if (a.adam) {
        e = launch_ex(rn_out_bwd, dim3(g), dim3(kT), 0, s, a.pdl != 0, a);
        if (e == cudaSuccess) e = launch_cluster(rn_blocks_bwd, a, s);
    }
    if (e == cudaSuccess) e = launch_ex(rn_in_step, dim3(g), dim3(kT), 0, s, a.pdl != 0, a);
    if (e == cudaSuccess) e = launch_cluster(rn_blocks_fwd, a, s);
    if (e == cudaSuccess) e = launch_ex(rn_out_fwd, dim3(g), dim3(kT), 0, s, a.pdl != 0, a);
    return e;
}
}  // namespace

// Step B of Algorithm 1 with the generator: one Adam step on theta from du,
// the forward pass to the new u, and the next waveform.
cudaError_t rn_enqueue_step(rn_net* n, const float* y0, const float* du, float* u, const long long* ctr, int inner,
                            int n_x, float lr, float b1, float b2, float eps, const QuantArgs& q, int next_wave,
                            float2* x_next, float* dydz_next, int pdl, cudaStream_t s) {
    RnArgs a = base_args(n);
    a.y0 = y0; a.du = du; a.u = u;
    a.adam = 1;
    a.lr = lr; a.b1 = b1; a.b2 = b2; a.eps = eps;
    a.ctr = ctr; a.inner = inner; a.n_x = n_x;
    a.q = q; a.next_wave = next_wave; a.x_next = x_next; a.dydz_next = dydz_next;
    a.pdl = pdl;
    return rn_enqueue(n, a, s);
}
int rn_size(const rn_net* n) { return n->P; }
}  // namespace af

extern "C" int64_t rn_param_count(int32_t P) {
    if (P < 1) return -1;
    return offsets(P).total;
}

extern "C" af_status rn_create(int32_t P, void* stream, rn_net** out) {
    if (!out) { g_rn_error = "out is NULL"; return AF_ERR_INVALID_ARG; }
    *out = nullptr;
    if (P < 1 || P > 65536) { g_rn_error = "P must be in 1..65536"; return AF_ERR_INVALID_ARG; }
    rn_net* n = new rn_net();
    n->P = P;
    n->o = offsets(P);
    n->stream = (cudaStream_t)stream;
    n->n_part = (P + kRB - 1) / kRB;
    const size_t T = (size_t)n->o.total;
    cudaError_t e = cudaMalloc(&n->th, sizeof(float) * T);
    if (e == cudaSuccess) e = cudaMalloc(&n->m, sizeof(float) * T);
    if (e == cudaSuccess) e = cudaMalloc(&n->v, sizeof(float) * T);
    if (e == cudaSuccess) e = cudaMalloc(&n->part, sizeof(float) * (size_t)n->n_part * kH);
    if (e == cudaSuccess) e = cudaMalloc(&n->hs, sizeof(float) * (kBlocks + 1) * kH);
    if (e == cudaSuccess) e = cudaMalloc(&n->rs, sizeof(float) * kBlocks * kH);
    if (e == cudaSuccess) e = cudaMalloc(&n->da, sizeof(float) * kH);
    if (e == cudaSuccess) e = cudaMalloc(&n->u, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMemset(n->th, 0, sizeof(float) * T);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, sizeof(float) * T);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, sizeof(float) * T);
    if (e != cudaSuccess) {
        g_rn_error = std::string("allocation: ") + cudaGetErrorString(e);
        rn_destroy(n);
        return e == cudaErrorMemoryAllocation ? AF_ERR_OOM : AF_ERR_CUDA;
    }
    *out = n;
    return AF_OK;
}

extern "C" af_status rn_destroy(rn_net* n) {
    if (!n) return AF_ERR_INVALID_ARG;
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (void* p : {(void*)n->th, (void*)n->m, (void*)n->v, (void*)n->part, (void*)n->hs, (void*)n->rs,
                    (void*)n->da, (void*)n->u})
        if (p) cudaFree(p);
    delete n;
    return AF_OK;
}

extern "C" const char* rn_last_error(const rn_net* n) { return n ? n->err.c_str() : g_rn_error.c_str(); }

extern "C" af_status rn_set_params(rn_net* n, const float* theta_host) {
    if (!n) return AF_ERR_INVALID_ARG;
    if (!theta_host) RN_FAIL(n, AF_ERR_INVALID_ARG, "rn_set_params: theta is NULL");
    const size_t T = (size_t)n->o.total;
    RN_CK(n, cudaStreamSynchronize(n->stream));
    RN_CK(n, cudaMemcpy(n->th, theta_host, sizeof(float) * T, cudaMemcpyHostToDevice));
    RN_CK(n, cudaMemset(n->m, 0, sizeof(float) * T));
    RN_CK(n, cudaMemset(n->v, 0, sizeof(float) * T));
    return AF_OK;
}

extern "C" af_status rn_get_params(rn_net* n, float* theta_host) {
    if (!n) return AF_ERR_INVALID_ARG;
    if (!theta_host) RN_FAIL(n, AF_ERR_INVALID_ARG, "rn_get_params: theta is NULL");
    RN_CK(n, cudaStreamSynchronize(n->stream));
    RN_CK(n, cudaMemcpy(theta_host, n->th, sizeof(float) * (size_t)n->o.total, cudaMemcpyDeviceToHost));
    return AF_OK;
}

extern "C" af_status rn_set_adam(rn_net* n, const float* m_host, const float* v_host) {
    if (!n) return AF_ERR_INVALID_ARG;
    if (!m_host || !v_host) RN_FAIL(n, AF_ERR_INVALID_ARG, "rn_set_adam: m and v must not be NULL");
    const size_t T = (size_t)n->o.total;
    RN_CK(n, cudaStreamSynchronize(n->stream));
    RN_CK(n, cudaMemcpy(n->m, m_host, sizeof(float) * T, cudaMemcpyHostToDevice));
    RN_CK(n, cudaMemcpy(n->v, v_host, sizeof(float) * T, cudaMemcpyHostToDevice));
    return AF_OK;
}

extern "C" af_status rn_get_adam(rn_net* n, float* m_host, float* v_host) {
    if (!n) return AF_ERR_INVALID_ARG;
    if (!m_host || !v_host) RN_FAIL(n, AF_ERR_INVALID_ARG, "rn_get_adam: m and v must not be NULL");
    const size_t T = (size_t)n->o.total;
    RN_CK(n, cudaStreamSynchronize(n->stream));
    RN_CK(n, cudaMemcpy(m_host, n->m, sizeof(float) * T, cudaMemcpyDeviceToHost));
    RN_CK(n, cudaMemcpy(v_host, n->v, sizeof(float) * T, cudaMemcpyDeviceToHost));
    return AF_OK;
}

extern "C" af_status rn_forward(rn_net* n, const float* y0_dev, float* u_dev) {
    if (!n) return AF_ERR_INVALID_ARG;
    if (!y0_dev || !u_dev) RN_FAIL(n, AF_ERR_INVALID_ARG, "rn_forward: y0 and u must not be NULL");
    RnArgs a = base_args(n);
    a.y0 = y0_dev;
    a.u = u_dev;
    a.adam = 0;
    a.next_wave = NEXT_NONE;
    RN_CK(n, rn_enqueue(n, a, n->stream));
    return AF_OK;
}

extern "C" af_status rn_train_step(rn_net* n, const float* y0_dev, const float* du_dev, float lr, int64_t t,
                                   float* u_dev) {
    if (!n) return AF_ERR_INVALID_ARG;
    if (!y0_dev || !du_dev || !u_dev) RN_FAIL(n, AF_ERR_INVALID_ARG, "rn_train_step: NULL pointer");
    if (t < 1 || !(lr >= 0.f)) RN_FAIL(n, AF_ERR_INVALID_ARG, "rn_train_step: t >= 1 and lr >= 0 required");
    RnArgs a = base_args(n);
    a.y0 = y0_dev;
    a.du = du_dev;
    a.u = u_dev;
    a.adam = 1;
    a.lr = lr;
    a.c1 = (float)(1.0 - pow(0.9, (double)t));
    a.c2 = (float)(1.0 - pow(0.999, (double)t));
    a.next_wave = NEXT_NONE;
    RN_CK(n, rn_enqueue(n, a, n->stream));
    return AF_OK;
}
