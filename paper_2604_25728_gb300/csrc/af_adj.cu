// af_adj.cu -- dense adjoint of the p-norm sidelobe loss on the FFT grid.
//
// With the smooth class value V = (sum_cells (w|chi|)^p)^(1/p) (the p-norm
// variant of Eqs. 8-9), every cell of the winning class carries
//     g(k, nu_j) = eps w (w|chi|/V)^(p-1) chi/|chi|,
// and the gradient of Eq. 42 is
//     grad x_m(n) += sum_{l,k} h_l(n+k) Gamma_{ml,k}(n)
//     grad h_l(p) += sum_{m,k} conj(Gamma_{ml,k}(p-k)) x_m(p-k)
// with Gamma(n) = sum_j g(k, nu_j) e^{-j 2 pi nu_j n}
//              = e^{-j 2 pi nu_0 n} conj(FFT+(conj g))(n mod L).
// The spectra chi are never stored: each CTA recomputes its rows with the
// forward FFT (the products are recomputed from x and h in shared memory),
// forms g in registers, runs a second FFT on conj(g) -- the forward FFT
// leaves its output in exactly the layout the next FFT reads -- and
// accumulates the two gradient rows of its pair in per-row-slot shared
// buffers, summed in a fixed order at the end (deterministic).  A second
// kernel sums the per-CTA partial rows.
#include "af_common.cuh"
#include "af_device.cuh"
#include "af_kernels.h"

namespace af {

constexpr int kAdjThreads = 256;

template <int L>
__host__ __device__ constexpr int adj_fold_len(int N) { return ((N + L - 1) / L) * L; }

// Merge the forward CTAs' p-norm partials of one class into the class value
// in the key domain: Vk^2 = vmax * s^(1/half_p) (Vk = V / w for uniform w).
__device__ float pnorm_class_key(const AdjArgs& a, int cls, float* shv, float* shs) {
    float v = 0.f, s = 0.f;
    for (int b = threadIdx.x; b < a.nblk_fwd; b += blockDim.x) {
        const int pair = b / a.ctas_per_pair_fwd;
        const int c = (pair / a.M == pair % a.M) ? 0 : 1;
        if (c == cls) pmerge(a.half_p, v, s, a.pvmax[b], a.psum[b]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const float os = __shfl_xor_sync(0xffffffffu, s, o);
        pmerge(a.half_p, v, s, ov, os);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { shv[threadIdx.x >> 5] = v; shs[threadIdx.x >> 5] = s; }
    __syncthreads();
    float vv = shv[0], ss = shs[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) pmerge(a.half_p, vv, ss, shv[w], shs[w]);
    return (vv > 0.f) ? vv * powf(ss, 1.f / a.half_p) : 0.f;
}

template <int L, int E>
__global__ void __launch_bounds__(kAdjThreads) adj_fft_kernel(const AdjArgs a) {
    using PL = Plan<L, E>;
    using C = float2;
    constexpr int TPR = PL::T;
    constexpr int RS = kAdjThreads / TPR;
    constexpr int RL = PL::radix(PL::passes - 1), NBL = E / RL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N;
    const int XS = adj_fold_len<L>(N);
    C* xs = reinterpret_cast<C*>(smem_raw);   // [XS] x e^{j 2 pi nu0 n}
    C* hp = xs + XS;                          // [2N + XS]
    C* tws = hp + 2 * N + XS;                 // [tw_len]
    C* bufs = tws + PL::tw_len;               // [RS][padlen]
    C* gxs = bufs + RS * PL::padlen;          // [RS][N] grad x_m partial per row slot
    C* ghs = gxs + RS * N;                    // [RS][N] grad h_l partial per row slot
    __shared__ float shv[kAdjThreads / 32], shs[kAdjThreads / 32];

    const int tid = threadIdx.x;
    const int pair = blockIdx.x / a.n_chunks;
    const int chunk = blockIdx.x - pair * a.n_chunks;
    const int m = pair / a.M, l = pair - m * a.M;
    const int my_cls = (m == l) ? 0 : 1;

    for (int i = tid; i < PL::tw_len; i += kAdjThreads) tws[i] = a.tw[i];
    pdl_wait();
    pdl_trigger();

    // the winning class (Eq. 37, auto on ties) and its value
    const float vk0 = pnorm_class_key(a, 0, shv, shs);
    const float vk1 = pnorm_class_key(a, 1, shv, shs);
    const float ws = (a.weight_mode == WM_UNIFORM) ? a.w0 : 1.f;
    const int cls = (ws * sqrtf(vk0) >= ws * sqrtf(vk1)) ? 0 : 1;
    const float vkey = (cls == 0) ? vk0 : vk1;
    C* out_x = a.part + (size_t)blockIdx.x * 2 * N;
    C* out_h = out_x + N;
    const C zero = make_float2(0.f, 0.f);
    if (my_cls != cls || !(vkey > 0.f)) {
        for (int i = tid; i < N; i += kAdjThreads) { out_x[i] = zero; out_h[i] = zero; }
        return;
    }
    const float inv_vkey = 1.f / vkey;
    const float expo = a.half_p - 0.5f;       // (w|chi|/V)^(p-1) = (key/Vk^2)^(p/2 - 1/2)

    for (int n = tid; n < XS; n += kAdjThreads) xs[n] = (n < N) ? cmul(a.x[(size_t)m * N + n], a.pre[n]) : zero;
    for (int i = tid; i < 2 * N + XS; i += kAdjThreads) {
        const int p = i - N;
        hp[i] = (p >= 0 && p < N) ? a.h[(size_t)l * N + p] : zero;
    }
    for (int i = tid; i < 2 * RS * N; i += kAdjThreads) gxs[i] = zero;
    __syncthreads();

    const int slot = tid / TPR;
    const int t = tid - slot * TPR;
    C* buf = bufs + slot * PL::padlen;
    C* gx_slot = gxs + slot * N;
    C* gh_slot = ghs + slot * N;
    const int d_begin = chunk * a.rows_per_chunk;
    const int d_end = min(a.D, d_begin + a.rows_per_chunk);
    const int NF = XS / L;

    for (int d0 = d_begin; d0 < d_end; d0 += RS) {
        const int d = d0 + slot;
        const bool row_in = d < d_end;
        const int k = row_in ? a.k_lo + d : 0;
        const bool live = row_in && !(m == l && k == 0);
        // ---- recompute chi(k, .) exactly as the forward pass does ----
        C v[E];
        const C* xk = xs + t;
        const C* hk = hp + N + k + t;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            C q = zero;
            for (int c = 0; c < NF; ++c) q = cadd(q, cmulc(xk[r * TPR + c * L], hk[r * TPR + c * L]));
            v[r] = q;
        }
        pass_compute<L, E, E, 1>(v, t, tws);
        fft_rest<L, E, 1>(v, t, slot, buf, tws);
        // ---- g per bin, conjugated, into the input layout of the next FFT ----
        // bin of v[s*RL + r] is t + TPR*(s + r*NBL); the next pass 0 reads bin t + TPR*q as v2[q]
        C v2[E];
        const float* wrow = (row_in && a.weight_mode != WM_UNIFORM) ? a.wmap + (size_t)d * L + t : nullptr;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
#pragma unroll
            for (int s = 0; s < NBL; ++s) {
                const int q = s + r * NBL;
                const C c = v[s * RL + r];
                const float mag2 = c.x * c.x + c.y * c.y;
                float w = ws;
                if (wrow != nullptr) w = __ldg(wrow + TPR * q);
                const float key = (wrow != nullptr && a.weight_mode == WM_MAP) ? w * w * mag2 : mag2;
                float coef = 0.f;
                if (live && w > 0.f && mag2 > 0.f) {
                    // eps w (key/Vk^2)^(p/2 - 1/2) / |chi|
                    coef = (float)a.eps * w * exp2f(expo * __log2f(key * inv_vkey)) * rsqrtf(mag2);
                }
                v2[q] = make_float2(coef * c.x, -coef * c.y);   // conj(g)
            }
        }
        pass_compute<L, E, E, 1>(v2, t, tws);
        fft_rest<L, E, 1>(v2, t, slot, buf, tws);
        // ---- Gamma(n) = e^{-j 2 pi nu0 n} conj(v2) at n = t + TPR*q (+ c L) ----
        if (live) {
#pragma unroll
            for (int r = 0; r < RL; ++r) {
#pragma unroll
                for (int s = 0; s < NBL; ++s) {
                    const int q = s + r * NBL;
                    const C gt = v2[s * RL + r];
                    for (int c = 0; c < NF; ++c) {
                        const int n = t + TPR * q + c * L;
                        if (n >= N) break;
                        const int p = n + k;
                        if (p < 0 || p >= N) continue;
                        const C pre = a.pre[n];
                        // Gamma = conj(gt) * conj(pre) = conj(gt * pre)
                        const C gam = cconj(cmul(gt, pre));
                        gx_slot[n] = cadd(gx_slot[n], cmul(gam, hp[N + p]));
                        // x_m(n) = xs[n] * conj(pre[n])
                        gh_slot[p] = cadd(gh_slot[p], cmul(cconj(gam), cmulc(xs[n], pre)));
                    }
                }
            }
        }
        row_sync<TPR>(slot);
    }
    __syncthreads();
    // ---- fixed-order sum over row slots, one partial row each for x_m and h_l ----
    for (int i = tid; i < N; i += kAdjThreads) {
        C sx = zero, sh = zero;
        for (int r = 0; r < RS; ++r) { sx = cadd(sx, gxs[r * N + i]); sh = cadd(sh, ghs[r * N + i]); }
        out_x[i] = sx;
        out_h[i] = sh;
    }
}

// grad x_r(n) = sum over pairs (r, l) and chunks; grad h_r(n) over pairs (m, r).
__global__ void adj_reduce_kernel(const AdjArgs a) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y, which = blockIdx.z;
    pdl_wait();
    pdl_trigger();
    if (n >= a.N) return;
    float2 acc = make_float2(0.f, 0.f);
    for (int o = 0; o < a.M; ++o) {
        const int pair = (which == 0) ? r * a.M + o : o * a.M + r;
        for (int c = 0; c < a.n_chunks; ++c) {
            const size_t cta = (size_t)pair * a.n_chunks + c;
            acc = cadd(acc, a.part[cta * 2 * a.N + (size_t)which * a.N + n]);
        }
    }
    a.dense[(size_t)which * a.M * a.N + (size_t)r * a.N + n] = acc;
}

template <int L, int E>
static int adj_smem(int N) {
    using PL = Plan<L, E>;
    const int XS = adj_fold_len<L>(N);
    const int RS = kAdjThreads / PL::T;
    return (int)sizeof(float2) * (XS + 2 * N + XS + PL::tw_len + RS * PL::padlen + 2 * RS * N);
}

template <int L, int E>
static cudaError_t adj_launch_LE(const AdjArgs& a, cudaStream_t s, bool prepare_only) {
    const int smem = adj_smem<L, E>(a.N);
    auto kern = adj_fft_kernel<L, E>;
    cudaError_t e = set_smem_once(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess || prepare_only) return e;
    e = launch_ex(kern, dim3(a.M * a.M * a.n_chunks), dim3(kAdjThreads), smem, s, a.pdl != 0, a);
    if (e != cudaSuccess) return e;
    const dim3 rg((a.N + 255) / 256, a.M, 2);
    return launch_ex(adj_reduce_kernel, rg, dim3(256), 0, s, a.pdl != 0, a);
}

static cudaError_t adj_any(const AdjArgs& a, cudaStream_t s, bool prepare_only) {
    const bool e8 = (a.fft_e == 8);
    switch (a.L) {
        case 32: return e8 ? adj_launch_LE<32, 8>(a, s, prepare_only) : adj_launch_LE<32, 16>(a, s, prepare_only);
        case 64: return e8 ? adj_launch_LE<64, 8>(a, s, prepare_only) : adj_launch_LE<64, 16>(a, s, prepare_only);
        case 128: return e8 ? adj_launch_LE<128, 8>(a, s, prepare_only) : adj_launch_LE<128, 16>(a, s, prepare_only);
        case 256: return e8 ? adj_launch_LE<256, 8>(a, s, prepare_only) : adj_launch_LE<256, 16>(a, s, prepare_only);
        case 512: return e8 ? adj_launch_LE<512, 8>(a, s, prepare_only) : adj_launch_LE<512, 16>(a, s, prepare_only);
        case 1024: return e8 ? adj_launch_LE<1024, 8>(a, s, prepare_only) : adj_launch_LE<1024, 16>(a, s, prepare_only);
        case 2048: return e8 ? adj_launch_LE<2048, 8>(a, s, prepare_only) : adj_launch_LE<2048, 16>(a, s, prepare_only);
        case 4096: return e8 ? cudaErrorInvalidValue : adj_launch_LE<4096, 16>(a, s, prepare_only);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adj(const AdjArgs& a, cudaStream_t s) { return adj_any(a, s, false); }
cudaError_t adj_prepare(int L, int N, int E) {
    AdjArgs a{};
    a.L = L; a.N = N; a.fft_e = E;
    return adj_any(a, nullptr, true);
}
int adj_smem_bytes(int L, int N, int E) {
    if (E != 8 && E != 16) return -1;   // the adjoint is built for 8 and 16 values per thread
    const bool e8 = (E == 8);
    switch (L) {
        case 32: return e8 ? adj_smem<32, 8>(N) : adj_smem<32, 16>(N);
        case 64: return e8 ? adj_smem<64, 8>(N) : adj_smem<64, 16>(N);
        case 128: return e8 ? adj_smem<128, 8>(N) : adj_smem<128, 16>(N);
        case 256: return e8 ? adj_smem<256, 8>(N) : adj_smem<256, 16>(N);
        case 512: return e8 ? adj_smem<512, 8>(N) : adj_smem<512, 16>(N);
        case 1024: return e8 ? adj_smem<1024, 8>(N) : adj_smem<1024, 16>(N);
        case 2048: return e8 ? adj_smem<2048, 8>(N) : adj_smem<2048, 16>(N);
        case 4096: return e8 ? -1 : adj_smem<4096, 16>(N);
        default: return -1;
    }
}

}  // namespace af
