// af_fft.cu -- fused forward pass on a uniform Doppler grid nu_j = nu_0 + j/L.
//
// For every ordered pair (m, l) and delay k (Eq. 6, Eq. 34):
//   chi_ml(k, nu_j) = sum_n x_m(n) conj(h_l(n+k)) e^{j 2 pi nu_0 n} e^{+j 2 pi j n / L}
// i.e. an unnormalised inverse-sign L-point DFT of the lag products
// (folded modulo L when N > L, zero-padded when N < L).  One CTA owns one
// pair and a chunk of delays; x_m (pre-modulated by e^{j 2 pi nu_0 n}) and h_l
// sit in shared memory, each row's products are formed in registers and
// transformed by a Stockham FFT (radix 16/16/r, 16 values per thread, T = L/16
// threads per row, exchanges through a padded shared buffer).  The last pass
// leaves chi in registers, where the sidelobe reduction of Eqs. 7-9 runs:
// per-CTA max of w^2|chi|^2 with its lowest linear cell index, plus p-norm
// partials.  chi is never written to memory in the reduce mode.
//
// This replaces the zero-padded FFT correlation of Eq. 36 (Doppler-major:
// one FFT pair per Doppler bin) with a delay-major transform: one L-point FFT
// per (pair, delay) row, which is the form that keeps every operand on chip.
#include "af_common.cuh"
#include "af_kernels.h"

namespace af {

constexpr int kThreads = 256;

template <typename K>
__device__ __forceinline__ bool better(K a, long long ia, K b, long long ib) {
    return a > b || (a == b && ia < ib);
}

template <int L, typename C, typename K>
__global__ void __launch_bounds__(kThreads)
fwd_fft_kernel(const FwdArgs<C, K> a) {
    using PL = Plan<L>;
    using T = decltype(C{}.x);
    constexpr int TPR = PL::T;              // threads per row
    constexpr int RS = kThreads / TPR;       // row slots per CTA
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* xs = reinterpret_cast<C*>(smem_raw);
    C* hs = xs + a.N;
    C* tws = hs + a.N;
    C* bufs = tws + PL::tw_len;

    const int tid = threadIdx.x;
    if (a.ctr_inc != nullptr && blockIdx.x == 0 && tid == 0) a.ctr_inc[0] += 1;
    const int pair = blockIdx.x / a.n_chunks;
    const int chunk = blockIdx.x - pair * a.n_chunks;
    const int m = pair / a.M, l = pair - m * a.M;
    const int N = a.N;

    for (int n = tid; n < N; n += kThreads) {
        xs[n] = cmul(a.x[(size_t)m * N + n], a.pre[n]);
        hs[n] = a.h[(size_t)l * N + n];
    }
    for (int i = tid; i < PL::tw_len; i += kThreads) tws[i] = a.tw[i];

    // chi_mm(0, 0) = h_m^H x_m in FP64 (Eq. 38), once per waveform.
    if (a.cdiag != nullptr && m == l && chunk == 0) {
        double sr = 0.0, si = 0.0;
        for (int n = tid; n < N; n += kThreads) {
            C xv = a.x[(size_t)m * N + n], hv = a.h[(size_t)l * N + n];
            double xr = xv.x, xi = xv.y, hr = hv.x, hi = hv.y;
            sr += xr * hr + xi * hi;
            si += xi * hr - xr * hi;
        }
        __shared__ double red[2][kThreads / 32];
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if ((tid & 31) == 0) { red[0][tid >> 5] = sr; red[1][tid >> 5] = si; }
        __syncthreads();
        if (tid == 0) {
            double tr = 0, ti = 0;
            for (int w = 0; w < kThreads / 32; ++w) { tr += red[0][w]; ti += red[1][w]; }
            a.cdiag[m] = make_double2(tr, ti);
        }
    }
    __syncthreads();

    const int slot = tid / TPR;
    const int t = tid - slot * TPR;
    C* buf = bufs + slot * PL::padlen;
    const int d_begin = chunk * a.rows_per_chunk;
    const int d_end = min(a.D, d_begin + a.rows_per_chunk);

    K best = (K)-1;
    long long best_idx = 0x7fffffffffffffffLL;
    float pv = 0.f, ps = 0.f;                   // p-norm partials (key domain)
    const bool auto_pair = (m == l);

    for (int d0 = d_begin; d0 < d_end; d0 += RS) {
        const int d = d0 + slot;
        const bool row_in = d < d_end;
        const int k = a.k_lo + d;
        // ---- pass 0: lag products (folded mod L) + radix-16 butterflies ----
        C v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            C q = mk((T)0, (T)0);
            if (row_in) {
                for (int n = t + r * TPR; n < N; n += L) {
                    const int p = n + k;
                    if (p >= 0 && p < N) q = cadd(q, cmulc(xs[n], hs[p]));
                }
            }
            v[r] = q;
        }
        pass_compute<L, PL::radix(0), 1>(v, t, tws);
        fft_rest<L, 1>(v, t, slot, buf, tws);

        // ---- epilogue: chi(k, bin) is in registers ----
        constexpr int RL = PL::radix(PL::passes - 1);
        if (a.mode == FWD_DUMP) {
            if (row_in) {
                C* out = a.chi_out + ((size_t)pair * a.D + d) * L;
#pragma unroll
                for (int s = 0; s < 16 / RL; ++s)
#pragma unroll
                    for (int r = 0; r < RL; ++r) out[out_bin<L>(t, s, r)] = v[s * RL + r];
            }
        } else if (row_in && !(auto_pair && k == 0)) {
            const long long row_base = ((long long)pair * a.D + d) * L;
#pragma unroll
            for (int s = 0; s < 16 / RL; ++s) {
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    const int bin = out_bin<L>(t, s, r);
                    const C c = v[s * RL + r];
                    K key = (K)c.x * (K)c.x + (K)c.y * (K)c.y;
                    if (a.weight_mode != WM_UNIFORM) {
                        const float w = __ldg(a.wmap + (size_t)d * L + bin);
                        key = (w > 0.f) ? (a.weight_mode == WM_MAP ? (K)w * (K)w * key : key) : (K)-1;
                    }
                    const long long cell = row_base + bin;
                    if (better(key, cell, best, best_idx)) { best = key; best_idx = cell; }
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
        }
    }

    if (a.mode == FWD_DUMP) return;

    // ---- CTA reduction of (best, best_idx) and the p-norm partials ----
    for (int o = 16; o > 0; o >>= 1) {
        K ob = __shfl_xor_sync(0xffffffffu, best, o);
        long long oi = __shfl_xor_sync(0xffffffffu, best_idx, o);
        if (better(ob, oi, best, best_idx)) { best = ob; best_idx = oi; }
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
    __shared__ K rk[kThreads / 32];
    __shared__ long long ri[kThreads / 32];
    __shared__ float rv[kThreads / 32], rsum[kThreads / 32];
    const int warp = tid >> 5;
    if ((tid & 31) == 0) { rk[warp] = best; ri[warp] = best_idx; rv[warp] = pv; rsum[warp] = ps; }
    __syncthreads();
    if (tid == 0) {
        K b = rk[0];
        long long bi = ri[0];
        float vv = rv[0], ss = rsum[0];
        for (int w = 1; w < kThreads / 32; ++w) {
            if (better(rk[w], ri[w], b, bi)) { b = rk[w]; bi = ri[w]; }
            if (a.half_p > 0.f) {
                float nv = fmaxf(vv, rv[w]);
                float sa = (vv > 0.f) ? ss * exp2f(a.half_p * __log2f(vv / nv)) : 0.f;
                float sb = (rv[w] > 0.f) ? rsum[w] * exp2f(a.half_p * __log2f(rv[w] / nv)) : 0.f;
                vv = nv;
                ss = sa + sb;
            }
        }
        a.pkey[blockIdx.x] = b;
        a.pidx[blockIdx.x] = (b >= (K)0) ? bi : -1;
        if (a.pvmax) { a.pvmax[blockIdx.x] = vv; a.psum[blockIdx.x] = ss; }
    }
}

template <int L, typename C, typename K>
static int smem_for(int N) {
    return (int)sizeof(C) * (2 * N + Plan<L>::tw_len + (kThreads / Plan<L>::T) * Plan<L>::padlen);
}

template <int L, typename C, typename K>
static cudaError_t launch_L(const FwdArgs<C, K>& a, cudaStream_t s) {
    const int smem = smem_for<L, C, K>(a.N);
    auto kern = fwd_fft_kernel<L, C, K>;
    cudaError_t e = set_smem_once(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
    const int grid = a.M * a.M * a.n_chunks;
    kern<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int L, typename C, typename K>
static cudaError_t prepare_L(int N) {
    return set_smem_once(reinterpret_cast<const void*>(fwd_fft_kernel<L, C, K>), smem_for<L, C, K>(N));
}

template <typename C, typename K>
static cudaError_t prepare_any(int L, int N) {
    switch (L) {
        case 32: return prepare_L<32, C, K>(N);
        case 64: return prepare_L<64, C, K>(N);
        case 128: return prepare_L<128, C, K>(N);
        case 256: return prepare_L<256, C, K>(N);
        case 512: return prepare_L<512, C, K>(N);
        case 1024: return prepare_L<1024, C, K>(N);
        case 2048: return prepare_L<2048, C, K>(N);
        case 4096: return prepare_L<4096, C, K>(N);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fft_prepare_f32(int L, int N) { return prepare_any<float2, float>(L, N); }
cudaError_t fft_prepare_f64(int L, int N) { return prepare_any<double2, double>(L, N); }

template <typename C, typename K>
static cudaError_t launch_any(const FwdArgs<C, K>& a, cudaStream_t s) {
    switch (a.L) {
        case 32: return launch_L<32>(a, s);
        case 64: return launch_L<64>(a, s);
        case 128: return launch_L<128>(a, s);
        case 256: return launch_L<256>(a, s);
        case 512: return launch_L<512>(a, s);
        case 1024: return launch_L<1024>(a, s);
        case 2048: return launch_L<2048>(a, s);
        case 4096: return launch_L<4096>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fwd_fft_f32(const FwdArgs<float2, float>& a, cudaStream_t s) { return launch_any(a, s); }
cudaError_t launch_fwd_fft_f64(const FwdArgs<double2, double>& a, cudaStream_t s) { return launch_any(a, s); }

template <typename C>
static int smem_any(int L, int N) {
    switch (L) {
        case 32: return smem_for<32, C, float>(N);
        case 64: return smem_for<64, C, float>(N);
        case 128: return smem_for<128, C, float>(N);
        case 256: return smem_for<256, C, float>(N);
        case 512: return smem_for<512, C, float>(N);
        case 1024: return smem_for<1024, C, float>(N);
        case 2048: return smem_for<2048, C, float>(N);
        case 4096: return smem_for<4096, C, float>(N);
        default: return -1;
    }
}

int fft_smem_bytes(int L, int N, bool fp64) { return fp64 ? smem_any<double2>(L, N) : smem_any<float2>(L, N); }

int fft_rows_per_cta(int L) { return (L >= 32 && L <= 4096) ? kThreads / (L / 16) : 0; }

int fft_tw_len(int L) {
    switch (L) {
        case 32: return Plan<32>::tw_len;
        case 64: return Plan<64>::tw_len;
        case 128: return Plan<128>::tw_len;
        case 256: return Plan<256>::tw_len;
        case 512: return Plan<512>::tw_len;
        case 1024: return Plan<1024>::tw_len;
        case 2048: return Plan<2048>::tw_len;
        case 4096: return Plan<4096>::tw_len;
        default: return -1;
    }
}

}  // namespace af
