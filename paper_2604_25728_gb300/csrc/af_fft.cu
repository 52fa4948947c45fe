// af_fft.cu -- fused forward pass on a uniform Doppler grid nu_j = nu_0 + j/L.
//
// For every ordered pair (m, l) and delay k (Eq. 6, Eq. 34):
//   chi_ml(k, nu_j) = sum_n x_m(n) conj(h_l(n+k)) e^{j 2 pi nu_0 n} e^{+j 2 pi j n / L}
// i.e. an unnormalised inverse-sign L-point DFT of the lag products
// (folded modulo L when N > L, zero-padded when N < L).  One CTA of NT
// threads owns one pair and a chunk of delays.  x_m (pre-modulated by
// e^{j 2 pi nu_0 n}, zero beyond N) and the window of h_l that the chunk's
// delays reach (zero outside [0, N)) sit in shared memory, so each row's
// products are formed in registers without bounds checks.  The row is
// transformed by a Stockham FFT with E values per thread (T = L/E threads per
// row, radix E passes then the remainder, exchanges through a padded shared
// buffer; at L = 2048, E = 32 the last radix-2 pass is paired across the
// row's two warps and exchanges half the data).  The last pass leaves chi in
// registers, where the sidelobe reduction of Eqs. 7-9 runs: per-CTA max of
// w^2|chi|^2 with its lowest linear cell index, plus p-norm partials.  chi
// is never written to memory in the reduce modes.
//
// This replaces the zero-padded FFT correlation of Eq. 36 (Doppler-major:
// one FFT pair per Doppler bin) with a delay-major transform: one L-point FFT
// per (pair, delay) row, which is the form that keeps every operand on chip.
#include <stdlib.h>

#include <type_traits>
#include <vector>

#include "af_common.cuh"
#include "af_kernels.h"

namespace af {

enum : int { MODE_REDUCE = 0, MODE_REDUCE_PNORM = 1, MODE_DUMP = 2 };

template <typename K>
__device__ __forceinline__ bool better(K a, long long ia, K b, long long ib) {
    return a > b || (a == b && ia < ib);
}

__device__ __forceinline__ void pnorm_merge(float hp, float& pv, float& ps, float ov, float os) {
    const float nv = fmaxf(pv, ov);
    const float sa = (pv > 0.f) ? ps * exp2f(hp * __log2f(pv / nv)) : 0.f;
    const float sb = (ov > 0.f) ? os * exp2f(hp * __log2f(ov / nv)) : 0.f;
    pv = nv;
    ps = sa + sb;
}

template <int L>
__host__ __device__ constexpr int fold_len(int N) { return ((N + L - 1) / L) * L; }

// Shared-memory entries of one CTA: x (XS), the h window (XS + rows per
// chunk), the twiddles and RS padded row buffers.
template <int L, int E, int NT>
__host__ __device__ constexpr int fft_smem_entries(int N, int rpc) {
    return fold_len<L>(N) * 2 + rpc + Plan<L, E>::tw_len + (NT / (L / E)) * Plan<L, E>::padlen;
}

// The last pass of a 2048-point row at 32 values per thread (passes 32, 32,
// 2; the row's 64 threads are two warps).  After pass 1, lane l of warp h
// holds in register r the element l + 32 r + 1024 h, so the radix-2
// butterfly x = l + 32 r (NS = 1024) pairs register r of lane l in the two
// warps.  Warp 0 takes r < 16 and warp 1 r >= 16: each warp hands its
// partner lane the 16 registers the partner keeps -- half the data of a full
// exchange -- through warp-uniform branches with compile-time register
// indices.  Leaves y(x) in v[q] and y(x + 1024) in v[16 + q] for
// x = l + 32 (q + 16 h).
template <typename C>
__device__ __forceinline__ void last_pass_pair(C (&v)[32], int t, int slot, C* buf, const C* tw_last) {
    const int l = t & 31, h = t >> 5;
    C w[16];
    if (h == 0) {
#pragma unroll
        for (int q = 0; q < 16; ++q) buf[q * 64 + l] = v[16 + q];
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) buf[q * 64 + 32 + l] = v[q];
    }
    row_sync<64>(slot);
    if (h == 0) {
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = buf[q * 64 + 32 + l];
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = buf[q * 64 + l];
    }
    row_sync<64>(slot);
    if (h == 0) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const C b = cmul(w[q], tw_last[l + 32 * q]);
            const C a = v[q];
            v[q] = padd(a, b);
            v[16 + q] = psub(a, b);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const C b = cmul(v[16 + q], tw_last[l + 32 * (16 + q)]);
            const C a = w[q];
            v[q] = padd(a, b);
            v[16 + q] = psub(a, b);
        }
    }
}

// Cell i (0 <= i < E) of a thread's row after the last pass, in increasing
// bin order: its register and its bin relative to the thread's first bin.
template <int E, int TPR, int RL, int NBL, int NSL, bool PAIR>
struct CellMap {
    static __device__ __forceinline__ constexpr int reg(int i) { return PAIR ? i : (i % NBL) * RL + i / NBL; }
    static __device__ __forceinline__ constexpr int off(int i) {
        return PAIR ? 32 * (i % 16) + 1024 * (i / 16) : TPR * (i % NBL) + (i / NBL) * NSL;
    }
};

// FP32 CTAs of 256 threads keep to 128 registers, so that two fit on an SM
// when their shared memory allows.
template <int L, int E, int NT, int MODE, typename C, typename K>
__global__ void __launch_bounds__(NT, (NT == 256 && sizeof(C) == sizeof(float2)) ? 2 : 1)
fwd_fft_kernel(const FwdArgs<C, K> a) {
    using PL = Plan<L, E>;
    using T = decltype(C{}.x);
    constexpr int kThreads = NT;
    constexpr int TPR = PL::T;               // threads per row
    constexpr int RS = kThreads / TPR;       // row slots per CTA
    constexpr int RL = PL::radix(PL::passes - 1), NSL = PL::ns(PL::passes - 1), NBL = E / RL;
    // rows of 2048 bins at 32 values per thread: the paired last pass
    constexpr bool kPair = (sizeof(C) == sizeof(float2) && L == 2048 && E == 32 && PL::passes == 3 && TPR == 64);
    using CM = CellMap<E, TPR, RL, NBL, NSL, kPair>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N;
    const int XS = fold_len<L>(N);
    const int HS = XS + a.rows_per_chunk;     // h window of this CTA's delays
    C* xs = reinterpret_cast<C*>(smem_raw);   // [XS]
    C* hs = xs + XS;                          // [HS], h_l(k_first + i) at hs[i]
    C* tws = hs + HS;                         // [tw_len]
    C* bufs = tws + PL::tw_len;               // [RS][padlen]

    const int tid = threadIdx.x;
    const int pair = blockIdx.x / a.n_chunks;
    const int chunk = blockIdx.x - pair * a.n_chunks;
    const int m = pair / a.M, l = pair - m * a.M;
    const int d_begin = chunk * a.rows_per_chunk;
    const int k_first = a.k_lo + d_begin;     // smallest delay of the chunk

    // Constant tables first: with programmatic launch this overlaps the tail
    // of the kernel that produces x and h.
    for (int i = tid; i < PL::tw_len; i += kThreads) tws[i] = a.tw[i];
    pdl_wait();
    pdl_trigger();
    if (a.ctr_inc != nullptr && blockIdx.x == 0 && tid == 0) a.ctr_inc[0] += 1;

    const C zero = mk((T)0, (T)0);
    // operand fill: every load of a batch is in flight before the first store
    {
        constexpr int FB = 4;
        const C* xm = a.x + (size_t)m * N;
        const C* hl = a.h + (size_t)l * N;
        for (int n0 = tid; n0 < XS; n0 += kThreads * FB) {
            C xv[FB], pv[FB];
#pragma unroll
            for (int q = 0; q < FB; ++q) {
                const int n = n0 + q * kThreads;
                xv[q] = (n < N) ? xm[n] : zero;
                pv[q] = (n < N) ? a.pre[n] : zero;
            }
#pragma unroll
            for (int q = 0; q < FB; ++q) {
                const int n = n0 + q * kThreads;
                if (n < XS) xs[n] = cmul(xv[q], pv[q]);
            }
        }
        // row k reads h_l(n + k) for n < XS: with k_first <= k < k_first +
        // rows_per_chunk that is hs[0 .. XS + rows_per_chunk - 1)
        for (int i0 = tid; i0 < HS; i0 += kThreads * FB) {
            C hv[FB];
#pragma unroll
            for (int q = 0; q < FB; ++q) {
                const int i = i0 + q * kThreads;
                const int p = k_first + i;
                hv[q] = (p >= 0 && p < N && i < HS) ? hl[p] : zero;
            }
#pragma unroll
            for (int q = 0; q < FB; ++q) {
                const int i = i0 + q * kThreads;
                if (i < HS) hs[i] = hv[q];
            }
        }
    }

    // chi_mm(0, 0) = h_m^H x_m (Eq. 38), once per waveform: double-float sums
    // in the FP32 instantiation, FP64 in the FP64 one.
    if constexpr (sizeof(K) == 4) {
        if (a.cdiag != nullptr && m == l && chunk == 0)
            diag_sum_f32<kThreads>(a.x + (size_t)m * N, a.h + (size_t)l * N, N, a.cdiag + m);
    } else if (a.cdiag != nullptr && m == l && chunk == 0) {
        double sr = 0.0, si = 0.0;
        for (int n = tid; n < N; n += kThreads) {
            const C xv = a.x[(size_t)m * N + n], hv = a.h[(size_t)l * N + n];
            const double xr = xv.x, xi = xv.y, hr = hv.x, hi = hv.y;
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
    const int d_end = min(a.D, d_begin + a.rows_per_chunk);
    const int NF = XS / L;
    const bool auto_pair = (m == l);

    K best = (K)-1;
    int best_li = 0;                          // (d - d_begin) * L + bin
    C best_c = zero;                          // chi at that cell
    float pv = 0.f, ps = 0.f, ipv = 0.f;      // p-norm partials (key domain): max key, sum of (key/pv)^hp, 1/pv

    for (int d0 = d_begin; d0 < d_end; d0 += RS) {
        const int d = d0 + slot;
        const bool row_in = d < d_end;
        const int k = row_in ? a.k_lo + d : k_first;   // rows past the chunk compute on valid data, unused
        // ---- pass 0: lag products (folded mod L) + radix-E butterflies ----
        C v[E];
        const C* xk = xs + t;
        const C* hk = hs + (k - k_first) + t;
        if (NF == 1) {
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = cmulc(xk[r * TPR], hk[r * TPR]);
        } else {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                C q = zero;
                for (int c = 0; c < NF; ++c) q = cadd(q, cmulc(xk[r * TPR + c * L], hk[r * TPR + c * L]));
                v[r] = q;
            }
        }
        pass_compute<L, E, E, 1>(v, t, tws);
        if constexpr (kPair) {
            pass_store<L, E, E, 1>(v, t, buf);
            row_sync<TPR>(slot);
            pass_load<L, E, E>(v, t, buf);
            row_sync<TPR>(slot);
            pass_compute<L, E, E, E>(v, t, tws + PL::tw_off(1));
            last_pass_pair(v, t, slot, buf, tws + PL::tw_off(2));
        } else {
            fft_rest<L, E, 1>(v, t, slot, buf, tws);
        }
        // this thread's first bin; cell i is bin cbase + CM::off(i), in v[CM::reg(i)]
        const int cbase = kPair ? (t & 31) + 512 * (t >> 5) : t;

        // ---- epilogue: chi(k, bin) is in registers, bins in increasing order ----
        if constexpr (MODE == MODE_DUMP) {
            if (row_in) {
                C* out = a.chi_out + ((size_t)pair * a.D + d) * L + cbase;
#pragma unroll
                for (int i = 0; i < E; ++i) out[CM::off(i)] = v[CM::reg(i)];
            }
        } else if (row_in && !(auto_pair && k == 0)) {
            const int lbase = (d - d_begin) * L + cbase;
            // The weighted scan is a separate copy of the loop: with the weight
            // test inside the unrolled loop the uniform path's instructions are
            // interleaved with the weighted ones and the hot loop spans twice
            // the instruction-cache lines.
            auto scan = [&](auto weighted) {
                const float* wrow = a.wmap + (size_t)d * L + cbase;
                if constexpr (!decltype(weighted)::value && sizeof(K) == 4 && (RL * NBL) % 8 == 0) {
                    // Uniform weights: the thread's cells in scan order (increasing
                    // cell index) in groups of 8.  A group only matters if its
                    // largest key beats the best so far, and then its first
                    // maximal cell is the candidate -- the same cell as a
                    // cell-by-cell scan with a strict comparison.
                    constexpr int GS = 8;
#pragma unroll
                    for (int g0 = 0; g0 < RL * NBL; g0 += GS) {
                        K key[GS];
#pragma unroll
                        for (int q = 0; q < GS; ++q) {
                            const C c = v[CM::reg(g0 + q)];
                            key[q] = (K)c.x * (K)c.x + (K)c.y * (K)c.y;
                        }
                        K gm = key[0];
#pragma unroll
                        for (int q = 1; q < GS; ++q) gm = fmaxf(gm, key[q]);
                        if (gm > best) {
                            // compile-time register indices only (a run-time index
                            // would move v to local memory)
                            int off = CM::off(g0 + GS - 1);
                            C cs = v[CM::reg(g0 + GS - 1)];
#pragma unroll
                            for (int q = GS - 2; q >= 0; --q)
                                if (key[q] == gm) {
                                    off = CM::off(g0 + q);
                                    cs = v[CM::reg(g0 + q)];
                                }
                            best = gm;
                            best_li = lbase + off;
                            best_c = cs;
                        }
                    }
                } else {
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const int off = CM::off(i);
                    const C c = v[CM::reg(i)];
                    K key = (K)c.x * (K)c.x + (K)c.y * (K)c.y;
                    if constexpr (decltype(weighted)::value) {
                        const float w = __ldg(wrow + off);
                        key = (w > 0.f) ? (a.weight_mode == WM_MAP ? (K)w * (K)w * key : key) : (K)-1;
                    }
                    if (key > best) { best = key; best_li = lbase + off; best_c = c; }
                }
                }
                if constexpr (MODE == MODE_REDUCE_PNORM) {
                    // the p-norm partial of this thread's cells of the row: their
                    // largest key first (one rescale of the running sum at most),
                    // then sum (key/pv)^hp with no branch per cell
                    float kmax = -1.f;
#pragma unroll
                    for (int i = 0; i < E; ++i) {
                        const C c = v[CM::reg(i)];
                        float key = (float)c.x * (float)c.x + (float)c.y * (float)c.y;
                        if constexpr (decltype(weighted)::value) {
                            const float w = __ldg(wrow + CM::off(i));
                            key = (w > 0.f) ? (a.weight_mode == WM_MAP ? w * w * key : key) : -1.f;
                        }
                        kmax = fmaxf(kmax, key);
                    }
                    if (kmax > pv) {
                        ps = (pv > 0.f) ? ps * exp2f(a.half_p * __log2f(pv / kmax)) : 0.f;
                        pv = kmax;
                        ipv = 1.f / kmax;
                    }
                    if (pv > 0.f) {
                        // (key/pv)^(p/2): p = 8 and 16 by squaring, other p by the
                        // hardware base-2 exponential and logarithm; one copy of the
                        // cell loop per kind (a uniform branch, none per cell)
                        auto sum_terms = [&](auto kind) {
                            constexpr int PK = decltype(kind)::value;
                            float acc = 0.f;
#pragma unroll
                            for (int i = 0; i < E; ++i) {
                                const C c = v[CM::reg(i)];
                                float key = (float)c.x * (float)c.x + (float)c.y * (float)c.y;
                                if constexpr (decltype(weighted)::value) {
                                    const float w = __ldg(wrow + CM::off(i));
                                    key = (w > 0.f) ? (a.weight_mode == WM_MAP ? w * w * key : key) : 0.f;
                                }
                                const float r = key * ipv;
                                if constexpr (PK == 4) {
                                    const float r2 = r * r;
                                    acc += r2 * r2;
                                } else if constexpr (PK == 8) {
                                    const float r2 = r * r, r4 = r2 * r2;
                                    acc += r4 * r4;
                                } else {
                                    acc += ex2_approx(a.half_p * __log2f(r));   // key = 0: log2 = -inf, a zero term
                                }
                            }
                            return acc;
                        };
                        if (a.half_p == 4.f) ps += sum_terms(std::integral_constant<int, 4>{});
                        else if (a.half_p == 8.f) ps += sum_terms(std::integral_constant<int, 8>{});
                        else ps += sum_terms(std::integral_constant<int, 0>{});
                    }
                }
            };
            if (a.weight_mode == WM_UNIFORM) scan(std::false_type{});
            else scan(std::true_type{});
        }
    }

    if constexpr (MODE != MODE_DUMP) {
        // ---- CTA reduction of (best, index) and the p-norm partials ----
        long long best_idx = (best >= (K)0) ? ((long long)pair * a.D + d_begin) * L + best_li
                                            : 0x7fffffffffffffffLL;
        for (int o = 16; o > 0; o >>= 1) {
            const K ob = __shfl_xor_sync(0xffffffffu, best, o);
            const long long oi = __shfl_xor_sync(0xffffffffu, best_idx, o);
            const T ocx = __shfl_xor_sync(0xffffffffu, best_c.x, o);
            const T ocy = __shfl_xor_sync(0xffffffffu, best_c.y, o);
            if (better(ob, oi, best, best_idx)) { best = ob; best_idx = oi; best_c = mk(ocx, ocy); }
            if constexpr (MODE == MODE_REDUCE_PNORM) {
                const float ov = __shfl_xor_sync(0xffffffffu, pv, o);
                const float os = __shfl_xor_sync(0xffffffffu, ps, o);
                pnorm_merge(a.half_p, pv, ps, ov, os);
            }
        }
        __shared__ K rk[kThreads / 32];
        __shared__ long long ri[kThreads / 32];
        __shared__ C rc[kThreads / 32];
        __shared__ float rv[kThreads / 32], rsum[kThreads / 32];
        const int warp = tid >> 5;
        if ((tid & 31) == 0) { rk[warp] = best; ri[warp] = best_idx; rc[warp] = best_c; rv[warp] = pv; rsum[warp] = ps; }
        __syncthreads();
        if (tid == 0) {
            K b = rk[0];
            long long bi = ri[0];
            C bc = rc[0];
            float vv = rv[0], ss = rsum[0];
            for (int w = 1; w < kThreads / 32; ++w) {
                if (better(rk[w], ri[w], b, bi)) { b = rk[w]; bi = ri[w]; bc = rc[w]; }
                if constexpr (MODE == MODE_REDUCE_PNORM) pnorm_merge(a.half_p, vv, ss, rv[w], rsum[w]);
            }
            a.pkey[blockIdx.x] = b;
            a.pidx[blockIdx.x] = (b >= (K)0) ? bi : -1;
            if (a.pchi) a.pchi[blockIdx.x] = bc;
            if (a.pvmax) { a.pvmax[blockIdx.x] = vv; a.psum[blockIdx.x] = ss; }
        }
    }
}

// ------------------------------------------------------------------ host ----
// A row needs L/E <= NT threads (one CTA).  E = 32 (one shared-memory
// exchange fewer, more registers) exists for the FP32 forward pass only; CTAs
// of 512 threads (twice the rows per CTA, sharing x, h and the twiddles) for
// FP32 rows of 1024 bins and more.
static bool shape_ok(int L, int E, int NT, bool fp64) {
    if (!(E == 8 || E == 16 || E == 32) || L < 2 * E || L / E > NT) return false;
    if (fp64) return E != 32 && NT == 256;
    return NT == 256 || (NT == 512 && E >= 16 && L >= 1024);
}

template <int L, int E, int NT, typename C>
static int smem_for(int N, int rpc) {
    return (int)sizeof(C) * fft_smem_entries<L, E, NT>(N, rpc);
}

template <int L, int E, int NT, int MODE, typename C, typename K>
static cudaError_t launch_LEM(const FwdArgs<C, K>& a, cudaStream_t s, bool prepare_only) {
    const int smem = smem_for<L, E, NT, C>(a.N, a.rows_per_chunk);
    auto kern = fwd_fft_kernel<L, E, NT, MODE, C, K>;
    cudaError_t e = set_smem_once(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess || prepare_only) return e;
    const int grid = a.M * a.M * a.n_chunks;
    return launch_ex(kern, dim3(grid), dim3(NT), smem, s, a.pdl != 0, a);
}

template <int L, int E, int NT, typename C, typename K>
static cudaError_t launch_LE(const FwdArgs<C, K>& a, cudaStream_t s, bool prepare_only) {
    if constexpr (sizeof(C) == sizeof(double2)) {
        // FP64 acceptance pass: exact max only
        return launch_LEM<L, E, NT, MODE_REDUCE, C, K>(a, s, prepare_only);
    } else {
        if (prepare_only) {
            cudaError_t e = launch_LEM<L, E, NT, MODE_REDUCE, C, K>(a, s, true);
            if (e == cudaSuccess) e = launch_LEM<L, E, NT, MODE_REDUCE_PNORM, C, K>(a, s, true);
            if (e == cudaSuccess) e = launch_LEM<L, E, NT, MODE_DUMP, C, K>(a, s, true);
            return e;
        }
        if (a.mode == FWD_DUMP) return launch_LEM<L, E, NT, MODE_DUMP, C, K>(a, s, false);
        if (a.half_p > 0.f) return launch_LEM<L, E, NT, MODE_REDUCE_PNORM, C, K>(a, s, false);
        return launch_LEM<L, E, NT, MODE_REDUCE, C, K>(a, s, false);
    }
}

// Every built (L, E, NT) instantiation, in one table: X(L, E, NT).
#define AF_FFT_F32_SHAPES(X)                                                                                 \
    X(32, 8, 256) X(32, 16, 256) X(64, 8, 256) X(64, 16, 256) X(64, 32, 256) X(128, 8, 256) X(128, 16, 256) \
    X(128, 32, 256) X(256, 8, 256) X(256, 16, 256) X(256, 32, 256) X(512, 8, 256) X(512, 16, 256)           \
    X(512, 32, 256) X(1024, 8, 256) X(1024, 16, 256) X(1024, 32, 256) X(2048, 8, 256) X(2048, 16, 256)      \
    X(2048, 32, 256) X(4096, 16, 256) X(4096, 32, 256) X(1024, 16, 512) X(1024, 32, 512) X(2048, 16, 512)    \
    X(2048, 32, 512) X(4096, 16, 512) X(4096, 32, 512)
#define AF_FFT_F64_SHAPES(X)                                                                                 \
    X(32, 8, 256) X(32, 16, 256) X(64, 8, 256) X(64, 16, 256) X(128, 8, 256) X(128, 16, 256) X(256, 8, 256)  \
    X(256, 16, 256) X(512, 8, 256) X(512, 16, 256) X(1024, 8, 256) X(1024, 16, 256) X(2048, 8, 256)         \
    X(2048, 16, 256) X(4096, 16, 256)

template <typename C, typename K>
static cudaError_t launch_any(const FwdArgs<C, K>& a, cudaStream_t s, bool prepare_only) {
    const int NT = a.fft_nt ? a.fft_nt : 256;
#define AF_FFT_CASE(LL, EE, TT) \
    if (a.L == LL && a.fft_e == EE && NT == TT) return launch_LE<LL, EE, TT>(a, s, prepare_only);
    if constexpr (sizeof(C) == sizeof(float2)) {
        AF_FFT_F32_SHAPES(AF_FFT_CASE)
    } else {
        AF_FFT_F64_SHAPES(AF_FFT_CASE)
    }
#undef AF_FFT_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_fwd_fft_f32(const FwdArgs<float2, float>& a, cudaStream_t s) { return launch_any(a, s, false); }
cudaError_t launch_fwd_fft_f64(const FwdArgs<double2, double>& a, cudaStream_t s) { return launch_any(a, s, false); }

template <int L, int E, int NT, typename C, typename K>
static int occupancy_LE(int N, int rpc) {
    // the occupancy query counts a launch above the kernel's shared-memory
    // limit as impossible, so the limit is raised first
    auto kern = fwd_fft_kernel<L, E, NT, MODE_REDUCE, C, K>;
    const int smem = smem_for<L, E, NT, C>(N, rpc);
    if (smem > 227 * 1024 || set_smem_once(reinterpret_cast<const void*>(kern), smem) != cudaSuccess) return 1;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess) return 1;
    return occ > 0 ? occ : 1;
}

int fft_occupancy(int L, int N, int E, bool fp64, int NT, int rpc) {
#define AF_FFT_OCC32(LL, EE, TT) \
    if (!fp64 && L == LL && E == EE && NT == TT) return occupancy_LE<LL, EE, TT, float2, float>(N, rpc);
#define AF_FFT_OCC64(LL, EE, TT) \
    if (fp64 && L == LL && E == EE && NT == TT) return occupancy_LE<LL, EE, TT, double2, double>(N, rpc);
    AF_FFT_F32_SHAPES(AF_FFT_OCC32)
    AF_FFT_F64_SHAPES(AF_FFT_OCC64)
#undef AF_FFT_OCC32
#undef AF_FFT_OCC64
    return 1;
}

cudaError_t fft_prepare_f32(int L, int N, int E, int NT, int rpc) {
    FwdArgs<float2, float> a{};
    a.L = L; a.N = N; a.fft_e = E; a.fft_nt = NT; a.rows_per_chunk = rpc;
    return launch_any(a, nullptr, true);
}
cudaError_t fft_prepare_f64(int L, int N, int E, int NT, int rpc) {
    FwdArgs<double2, double> a{};
    a.L = L; a.N = N; a.fft_e = E; a.fft_nt = NT; a.rows_per_chunk = rpc;
    return launch_any(a, nullptr, true);
}

int fft_rows_per_cta(int L, int E, int NT) { return (E > 0 && L % E == 0 && L / E <= NT) ? NT / (L / E) : 0; }

int fft_smem_bytes(int L, int N, bool fp64, int E, int NT, int rpc) {
    if (!shape_ok(L, E, NT, fp64) || (L & (L - 1)) != 0 || L > 4096) return -1;
    if (rpc <= 0) rpc = fft_rows_per_cta(L, E, NT);
    const int XS = ((N + L - 1) / L) * L;
    // the entries of fft_smem_entries, with the plan's table sizes
    int tw = 0, ns = 1, rem = L;
    std::vector<int> radices;
    while (rem >= E && rem % E == 0) { radices.push_back(E); rem /= E; }
    if (rem > 1) radices.push_back(rem);
    for (size_t p = 0; p < radices.size(); ++p) {
        if (p >= 1) tw += (radices[p] - 1) * ns;
        ns *= radices[p];
    }
    const long long entries = 2LL * XS + rpc + tw + (long long)(NT / (L / E)) * (L + L / E);
    const long long bytes = entries * (fp64 ? (long long)sizeof(double2) : (long long)sizeof(float2));
    return bytes > (1LL << 30) ? -1 : (int)bytes;
}

int fft_default_elems(int L, bool fp64) {
    if (const char* e = getenv("SQNGD_FFT_E")) {
        const int v = atoi(e);
        if (shape_ok(L, v, 256, fp64)) return v;
    }
    if (fp64) return shape_ok(L, 8, 256, true) ? 8 : 16;
    // rows of 512 bins and more: 32 values per thread save one shared-memory
    // exchange per row (measured 4-6% faster at L = 512 and 2048; slower for
    // short rows, where fewer CTAs fit)
    return (L >= 512 && shape_ok(L, 32, 256, false)) ? 32 : 16;
}

int fft_default_threads(int L, int E, bool fp64) {
    if (const char* e = getenv("SQNGD_FFT_NT")) {
        const int v = atoi(e);
        if (shape_ok(L, E, v, fp64)) return v;
    }
    // rows of 1024 bins and more with 32 values per thread: 512-thread CTAs
    // hold 16 warps per SM where the shared memory of 256-thread CTAs allows
    // one (measured at M=4, N=2048, L=2048: 326 -> 253 us per launch)
    return shape_ok(L, E, 512, fp64) && E == 32 ? 512 : 256;
}

}  // namespace af
