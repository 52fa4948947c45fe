// af_dft.cu -- forward pass on an arbitrary Doppler grid (SIMT, FP32 or FP64).
//
// chi[(pair, d), j] = sum_n P[(pair, d), n] E[n, j] with the lag products
// P = x_m(n) conj(h_l(n+k)) (Eq. 34) generated in shared memory from x and h,
// and E[n, j] = e^{j 2 pi nu_j n} an FP64-built phasor table.  One CTA owns a
// pair, 64 consecutive delays and 64 consecutive bins; each thread keeps a
// 4 x 4 block of complex accumulators.  The epilogue is the same sidelobe
// reduction as the FFT path (or a dump of chi).
#include "af_common.cuh"
#include "af_kernels.h"

namespace af {

constexpr int kDftThreads = 256;
constexpr int TR = 64;   // delays per CTA
constexpr int TC = 64;   // bins per CTA
constexpr int NK = 16;   // samples per shared-memory stage

template <typename K>
__device__ __forceinline__ bool dbetter(K a, long long ia, K b, long long ib) {
    return a > b || (a == b && ia < ib);
}

template <typename C, typename K>
__global__ void __launch_bounds__(kDftThreads)
fwd_dft_kernel(const FwdArgs<C, K> a) {
    using T = decltype(C{}.x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* xs = reinterpret_cast<C*>(smem_raw);
    C* hs = xs + a.N;
    C* As = hs + a.N;              // [NK][TR]
    C* Bs = As + NK * TR;          // [NK][TC]

    const int tid = threadIdx.x;
    pdl_wait();
    pdl_trigger();
    if (a.ctr_inc != nullptr && blockIdx.x == 0 && tid == 0) a.ctr_inc[0] += 1;
    const int n_ctiles = (a.L + TC - 1) / TC;
    const int bx = blockIdx.x;
    const int ctile = bx % n_ctiles;
    const int rest = bx / n_ctiles;
    const int pair = rest / a.n_chunks;
    const int chunk = rest - pair * a.n_chunks;
    const int m = pair / a.M, l = pair - m * a.M;
    const int N = a.N, L = a.L;
    const int d0 = chunk * TR, j0 = ctile * TC;

    for (int n = tid; n < N; n += kDftThreads) {
        xs[n] = a.x[(size_t)m * N + n];
        hs[n] = a.h[(size_t)l * N + n];
    }
    if constexpr (sizeof(K) == 4) {
        // double-float sums in the FP32 instantiation
        if (a.cdiag != nullptr && m == l && chunk == 0 && ctile == 0)
            diag_sum_f32<kDftThreads>(a.x + (size_t)m * N, a.h + (size_t)l * N, N, a.cdiag + m);
    } else if (a.cdiag != nullptr && m == l && chunk == 0 && ctile == 0) {
        double sr = 0.0, si = 0.0;
        for (int n = tid; n < N; n += kDftThreads) {
            C xv = a.x[(size_t)m * N + n], hv = a.h[(size_t)l * N + n];
            double xr = xv.x, xi = xv.y, hr = hv.x, hi = hv.y;
            sr += xr * hr + xi * hi;
            si += xi * hr - xr * hi;
        }
        __shared__ double red[2][kDftThreads / 32];
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if ((tid & 31) == 0) { red[0][tid >> 5] = sr; red[1][tid >> 5] = si; }
        __syncthreads();
        if (tid == 0) {
            double tr = 0, ti = 0;
            for (int w = 0; w < kDftThreads / 32; ++w) { tr += red[0][w]; ti += red[1][w]; }
            a.cdiag[m] = make_double2(tr, ti);
        }
    }
    __syncthreads();

    const int ty = tid / 16, tx = tid % 16;   // rows ty*4..+3, bins tx + 16*c
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = mk((T)0, (T)0);

    // Only samples n with some valid product in the tile are visited.
    const int k_first = a.k_lo + d0;
    const int k_last = a.k_lo + min(a.D, d0 + TR) - 1;
    const int n_begin = max(0, -k_last);
    const int n_end = min(N, N - k_first);
    for (int nb = n_begin; nb < n_end; nb += NK) {
        __syncthreads();
        for (int e = tid; e < NK * TR; e += kDftThreads) {
            const int nn = e / TR, rr = e - nn * TR;
            const int n = nb + nn, d = d0 + rr, k = a.k_lo + d, p = n + k;
            C q = mk((T)0, (T)0);
            if (n < n_end && d < a.D && p >= 0 && p < N) q = cmulc(xs[n], hs[p]);
            As[nn * TR + rr] = q;
        }
        for (int e = tid; e < NK * TC; e += kDftThreads) {
            const int nn = e / TC, cc = e - nn * TC;
            const int n = nb + nn, j = j0 + cc;
            Bs[nn * TC + cc] = (n < n_end && j < L) ? a.tw[(size_t)n * L + j] : mk((T)0, (T)0);
        }
        __syncthreads();
#pragma unroll 4
        for (int nn = 0; nn < NK; ++nn) {
            C av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[nn * TR + ty * 4 + i];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[nn * TC + tx + 16 * c];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[i][c].x = fma(av[i].x, bv[c].x, acc[i][c].x);
                    acc[i][c].x = fma(-av[i].y, bv[c].y, acc[i][c].x);
                    acc[i][c].y = fma(av[i].x, bv[c].y, acc[i][c].y);
                    acc[i][c].y = fma(av[i].y, bv[c].x, acc[i][c].y);
                }
        }
    }

    if (a.mode == FWD_DUMP) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int d = d0 + ty * 4 + i;
            if (d >= a.D) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + tx + 16 * c;
                if (j < L) a.chi_out[((size_t)pair * a.D + d) * L + j] = acc[i][c];
            }
        }
        return;
    }

    K best = (K)-1;
    long long best_idx = 0x7fffffffffffffffLL;
    C best_c = mk((T)0, (T)0);
    float pv = 0.f, ps = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int d = d0 + ty * 4 + i;
        const int k = a.k_lo + d;
        if (d >= a.D || (m == l && k == 0)) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j0 + tx + 16 * c;
            if (j >= L) continue;
            const C v = acc[i][c];
            K key = (K)v.x * (K)v.x + (K)v.y * (K)v.y;
            if (a.weight_mode != WM_UNIFORM) {
                const float w = __ldg(a.wmap + (size_t)d * L + j);
                key = (w > 0.f) ? (a.weight_mode == WM_MAP ? (K)w * (K)w * key : key) : (K)-1;
            }
            const long long cell = ((long long)pair * a.D + d) * L + j;
            if (dbetter(key, cell, best, best_idx)) { best = key; best_idx = cell; best_c = v; }
            if (a.half_p > 0.f && key >= (K)0) {
                const float kf = (float)key;
                if (kf > pv) {
                    ps = (pv > 0.f ? ps * exp2f(a.half_p * __log2f(pv / kf)) : 0.f) + 1.f;
                    pv = kf;
                } else if (pv > 0.f) {
                    ps += exp2f(a.half_p * __log2f(kf / pv));
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        K ob = __shfl_xor_sync(0xffffffffu, best, o);
        long long oi = __shfl_xor_sync(0xffffffffu, best_idx, o);
        const T ocx = __shfl_xor_sync(0xffffffffu, best_c.x, o);
        const T ocy = __shfl_xor_sync(0xffffffffu, best_c.y, o);
        if (dbetter(ob, oi, best, best_idx)) { best = ob; best_idx = oi; best_c = mk(ocx, ocy); }
        if (a.half_p > 0.f) {
            float ov = __shfl_xor_sync(0xffffffffu, pv, o);
            float os = __shfl_xor_sync(0xffffffffu, ps, o);
            float nv = fmaxf(pv, ov);
            float sa = (pv > 0.f) ? ps * exp2f(a.half_p * __log2f(pv / nv)) : 0.f;
            float sb = (ov > 0.f) ? os * exp2f(a.half_p * __log2f(ov / nv)) : 0.f;
            pv = nv;
            ps = sa + sb;
        }
    }
    __shared__ K rk[kDftThreads / 32];
    __shared__ long long ri[kDftThreads / 32];
    __shared__ C rc[kDftThreads / 32];
    __shared__ float rv[kDftThreads / 32], rsum[kDftThreads / 32];
    const int warp = tid >> 5;
    if ((tid & 31) == 0) { rk[warp] = best; ri[warp] = best_idx; rc[warp] = best_c; rv[warp] = pv; rsum[warp] = ps; }
    __syncthreads();
    if (tid == 0) {
        K b = rk[0];
        long long bi = ri[0];
        C bc = rc[0];
        float vv = rv[0], ss = rsum[0];
        for (int w = 1; w < kDftThreads / 32; ++w) {
            if (dbetter(rk[w], ri[w], b, bi)) { b = rk[w]; bi = ri[w]; bc = rc[w]; }
            if (a.half_p > 0.f) {
                float nv = fmaxf(vv, rv[w]);
                float sa = (vv > 0.f) ? ss * exp2f(a.half_p * __log2f(vv / nv)) : 0.f;
                float sb = (rv[w] > 0.f) ? rsum[w] * exp2f(a.half_p * __log2f(rv[w] / nv)) : 0.f;
                vv = nv;
                ss = sa + sb;
            }
        }
        a.pkey[bx] = b;
        a.pidx[bx] = (b >= (K)0) ? bi : -1;
        if (a.pchi) a.pchi[bx] = bc;
        if (a.pvmax) { a.pvmax[bx] = vv; a.psum[bx] = ss; }
    }
}

// ------------------------------------------------------------------------
// One Doppler bin (L = 1; nu = 0 is the zero-Doppler correlation of the
// paper's correlation experiments): chi_ml(k) = sum_n x'_m(n) conj(h_l(n+k))
// with x' = x e^{j 2 pi nu_0 n}, a plain cross-correlation.  The tiled DFT
// above would spend 63 of its 64 bin columns on padding, so this kernel
// gives each CTA 32 consecutive delays of one pair (lane = delay) and splits
// the samples n of their common range across its 16 warps.  Shared memory
// holds x' and h over that range, relative to its first sample and
// zero-padded, so lane t at offset i reads x'[i] (one broadcast) and
// h[i + t] (consecutive words): no bounds checks, no bank conflicts.  The
// warps' partial sums are added in a fixed order by warp 0, which also
// runs the sidelobe reduction of its 32 cells.
constexpr int kCorrThreads = 512;
constexpr int kCorrWarps = kCorrThreads / 32;
constexpr int TRC = 32;            // delays per CTA
constexpr int kCorrPad = 4 * kCorrWarps + TRC;   // extra slots beyond N in each buffer

template <typename C, typename K>
__global__ void __launch_bounds__(kCorrThreads)
fwd_corr_kernel(const FwdArgs<C, K> a) {
    using T = decltype(C{}.x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N;
    C* xs = reinterpret_cast<C*>(smem_raw);      // [N + kCorrPad]
    C* hs = xs + N + kCorrPad;                   // [N + 2 kCorrPad]
    __shared__ C red[kCorrWarps][TRC];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_wait();
    pdl_trigger();
    if (a.ctr_inc != nullptr && blockIdx.x == 0 && tid == 0) a.ctr_inc[0] += 1;
    const int pair = blockIdx.x / a.n_chunks;
    const int chunk = blockIdx.x - pair * a.n_chunks;
    const int m = pair / a.M, l = pair - m * a.M;
    const int d0 = chunk * TRC;
    const int k_first = a.k_lo + d0;
    const int k_last = a.k_lo + min(a.D, d0 + TRC) - 1;
    // samples with some valid product in this chunk
    const int n_begin = max(0, -k_last);
    const int n_end = min(N, N - k_first);
    const int len = n_end - n_begin;                       // >= 1 for any delay in -(N-1)..N-1
    const int S4 = 4 * ((len + 4 * kCorrWarps - 1) / (4 * kCorrWarps));   // samples per warp
    const int span = kCorrWarps * S4;                      // < len + kCorrPad - TRC
    const C* xg = a.x + (size_t)m * N;
    const C* hg = a.h + (size_t)l * N;
    for (int i = tid; i < span; i += kCorrThreads) {
        const int n = n_begin + i;
        xs[i] = (n < n_end) ? cmul(xg[n], a.tw[n]) : mk((T)0, (T)0);
    }
    const int p_lo = n_begin + k_first;
    for (int q = tid; q < span + TRC; q += kCorrThreads) {
        const int p = p_lo + q;
        hs[q] = (p >= 0 && p < N) ? hg[p] : mk((T)0, (T)0);
    }
    // A_mm(0, 0) (Eq. 38): double-float sums in the FP32 instantiation, FP64 in the FP64 one
    if constexpr (sizeof(K) == 4) {
        if (a.cdiag != nullptr && m == l && chunk == 0) diag_sum_f32<kCorrThreads>(xg, hg, N, a.cdiag + m);
    } else if (a.cdiag != nullptr && m == l && chunk == 0) {
        double sr = 0.0, si = 0.0;
        for (int n = tid; n < N; n += kCorrThreads) {
            const C xv = xg[n], hv = hg[n];
            const double xr = xv.x, xi = xv.y, hr = hv.x, hi = hv.y;
            sr += xr * hr + xi * hi;
            si += xi * hr - xr * hi;
        }
        __shared__ double rd[2][kCorrWarps];
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) { rd[0][warp] = sr; rd[1][warp] = si; }
        __syncthreads();
        if (tid == 0) {
            double tr = 0.0, ti = 0.0;
            for (int w = 0; w < kCorrWarps; ++w) { tr += rd[0][w]; ti += rd[1][w]; }
            a.cdiag[m] = make_double2(tr, ti);
        }
    }
    __syncthreads();

    // lane = delay k_first + lane, warp = samples [warp S4, (warp + 1) S4) of the range
    C acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = mk((T)0, (T)0);
    const int i0 = warp * S4;
    for (int i = i0; i < i0 + S4; i += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const C xv = xs[i + u];
            const C hv = hs[i + u + lane];
            acc[u].x = fma(xv.x, hv.x, acc[u].x);
            acc[u].x = fma(xv.y, hv.y, acc[u].x);
            acc[u].y = fma(xv.y, hv.x, acc[u].y);
            acc[u].y = fma(-xv.x, hv.y, acc[u].y);
        }
    }
    red[warp][lane] = cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
    __syncthreads();
    if (warp != 0) return;
    C v = red[0][lane];
#pragma unroll
    for (int w = 1; w < kCorrWarps; ++w) v = cadd(v, red[w][lane]);
    const int d = d0 + lane;
    if (a.mode == FWD_DUMP) {
        if (d < a.D) a.chi_out[(size_t)pair * a.D + d] = v;
        return;
    }
    K key = (K)-1;
    if (d < a.D && !(m == l && a.k_lo + d == 0)) {
        key = (K)v.x * (K)v.x + (K)v.y * (K)v.y;
        if (a.weight_mode != WM_UNIFORM) {
            const float w = __ldg(a.wmap + d);
            key = (w > 0.f) ? (a.weight_mode == WM_MAP ? (K)w * (K)w * key : key) : (K)-1;
        }
    }
    long long idx = (key >= (K)0) ? (long long)pair * a.D + d : 0x7fffffffffffffffLL;
    C bc = v;
    for (int o = 16; o > 0; o >>= 1) {
        const K ok = __shfl_xor_sync(0xffffffffu, key, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, idx, o);
        const T ocx = __shfl_xor_sync(0xffffffffu, bc.x, o);
        const T ocy = __shfl_xor_sync(0xffffffffu, bc.y, o);
        if (dbetter(ok, oi, key, idx)) { key = ok; idx = oi; bc = mk(ocx, ocy); }
    }
    if (lane == 0) {
        a.pkey[blockIdx.x] = key;
        a.pidx[blockIdx.x] = (key >= (K)0) ? idx : -1;
        if (a.pchi) a.pchi[blockIdx.x] = bc;
        if (a.pvmax) { a.pvmax[blockIdx.x] = 0.f; a.psum[blockIdx.x] = 0.f; }
    }
}

template <typename C>
static int corr_smem_bytes(int N) { return (int)sizeof(C) * (2 * N + 3 * kCorrPad); }

template <typename C, typename K>
static cudaError_t launch_dft(const FwdArgs<C, K>& a, cudaStream_t s) {
    if (a.L == 1) {
        const int smem = corr_smem_bytes<C>(a.N);
        auto kern = fwd_corr_kernel<C, K>;
        cudaError_t e = set_smem_once(reinterpret_cast<const void*>(kern), smem);
        if (e != cudaSuccess) return e;
        return launch_ex(kern, dim3(a.M * a.M * a.n_chunks), dim3(kCorrThreads), smem, s, a.pdl != 0, a);
    }
    const int smem = (int)sizeof(C) * (2 * a.N + NK * TR + NK * TC);
    auto kern = fwd_dft_kernel<C, K>;
    cudaError_t e = set_smem_once(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
    const int n_ctiles = (a.L + TC - 1) / TC;
    const int grid = a.M * a.M * a.n_chunks * n_ctiles;
    return launch_ex(kern, dim3(grid), dim3(kDftThreads), smem, s, a.pdl != 0, a);
}

template <typename C, typename K>
static cudaError_t prepare_dft(int N) {
    const int smem = (int)sizeof(C) * (2 * N + NK * TR + NK * TC);
    cudaError_t e = set_smem_once(reinterpret_cast<const void*>(fwd_dft_kernel<C, K>), smem);
    if (e != cudaSuccess) return e;
    return set_smem_once(reinterpret_cast<const void*>(fwd_corr_kernel<C, K>), corr_smem_bytes<C>(N));
}

cudaError_t dft_prepare_f32(int N) { return prepare_dft<float2, float>(N); }
cudaError_t dft_prepare_f64(int N) { return prepare_dft<double2, double>(N); }

int dft_rows_per_cta(int L) { return L == 1 ? TRC : TR; }
int dft_col_tiles(int L) { return (L + TC - 1) / TC; }

cudaError_t launch_fwd_dft_f32(const FwdArgs<float2, float>& a, cudaStream_t s) { return launch_dft(a, s); }
cudaError_t launch_fwd_dft_f64(const FwdArgs<double2, double>& a, cudaStream_t s) { return launch_dft(a, s); }

}  // namespace af
