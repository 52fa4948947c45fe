// af_adj.cu -- dense adjoint of the p-norm sidelobe loss on the FFT grid.
//
// With the smooth class value V = (sum_cells (w|chi|)^p)^(1/p) (the p-norm
// variant of Eqs. 8-9), every cell of the winning class carries
//     g(k, nu_j) = eps w (w|chi|/V)^(p-1) chi/|chi|,
// and the gradient of Eq. 42 is
//     grad x_m(n) += sum_{l,k} h_l(n+k) Gamma_{ml,k}(n)
//     grad h_l(p) += sum_{m,k} conj(Gamma_{ml,k}(p-k)) x_m(p-k)
// with Gamma(n) = sum_j g(k, nu_j) e^{-j 2 pi nu_j n}
//              = e^{-j 2 pi nu_0 n} conj(G2(n mod L)),  G2 = FFT+(conj g).
// With xs(n) = x_m(n) e^{j 2 pi nu_0 n} (the forward pass's operand) the two
// sums need no phase factor inside the loop over delays:
//     grad h_l(n+k) += G2(n) xs(n)
//     grad x_m(n)   += e^{-j 2 pi nu_0 n} sum_k conj(G2(n)) h_l(n+k)
// (the phase of the second is applied once per sample at the end).
//
// The spectra chi are never stored: each CTA recomputes its rows with the
// forward FFT (the products are recomputed from x and the h window in shared
// memory), forms g in registers, runs a second FFT on conj(g) -- the forward
// FFT leaves its output in exactly the layout the next FFT reads -- and
// accumulates.  A thread owns the same samples n of every row it transforms,
// so grad x accumulates in registers (rows of L >= N bins); grad h moves with
// the delay and accumulates in a shared row per row slot.  The grid covers
// only the winning class: CTA b takes chunk b mod c of pair b / c of that
// class, with the chunk counts c per class chosen on the host so that both
// classes fill the same grid.  Partial rows are summed in a fixed order by a
// second kernel (deterministic).
#include <type_traits>

#include "af_common.cuh"
#include "af_device.cuh"
#include "af_kernels.h"

namespace af {

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

// Pair (m, l) of index pi within class cls: the M auto pairs (m, m), or the
// M (M - 1) cross pairs in row-major order with the diagonal skipped.
__host__ __device__ __forceinline__ void class_pair(int cls, int pi, int M, int& m, int& l) {
    if (cls == 0) { m = l = pi; return; }
    m = pi / (M - 1);
    const int lp = pi - m * (M - 1);
    l = lp + (lp >= m ? 1 : 0);
}

// Shared-memory entries: xs (XS), the h window (XS + rows), the twiddles, RS
// padded row buffers, RS grad h rows, and (rows folded modulo L, N > L) RS
// grad x rows.
template <int L, int E, int NT>
__host__ __device__ constexpr int adj_smem_entries(int N, int rpc) {
    return adj_fold_len<L>(N) * 2 + rpc + Plan<L, E>::tw_len + (NT / (L / E)) * Plan<L, E>::padlen +
           (NT / (L / E)) * N * (N > L ? 2 : 1);
}

template <int L, int E, int NT>
__global__ void __launch_bounds__(NT, 1) adj_fft_kernel(const AdjArgs a) {
    using PL = Plan<L, E>;
    using C = float2;
    constexpr int TPR = PL::T;
    constexpr int RS = NT / TPR;
    constexpr int RL = PL::radix(PL::passes - 1), NBL = E / RL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, M = a.M;
    const int XS = adj_fold_len<L>(N);
    const int HS = XS + a.rpc_max;
    const int NF = XS / L;
    C* xs = reinterpret_cast<C*>(smem_raw);   // [XS] x e^{j 2 pi nu0 n}, zero beyond N
    C* hs = xs + XS;                          // [HS] h_l(k_first + i)
    C* tws = hs + HS;                         // [tw_len]
    C* bufs = tws + PL::tw_len;               // [RS][padlen]
    C* ghs = bufs + RS * PL::padlen;          // [RS][N] grad h_l partial per row slot
    C* gxs = ghs + RS * N;                    // [RS][N] grad x_m partial per row slot (N > L only)
    __shared__ float shv[NT / 32], shs[NT / 32];

    const int tid = threadIdx.x;
    for (int i = tid; i < PL::tw_len; i += NT) tws[i] = a.tw[i];
    pdl_wait();
    pdl_trigger();

    // the winning class (Eq. 37, auto on ties) and its value
    const float vk0 = pnorm_class_key(a, 0, shv, shs);
    const float vk1 = pnorm_class_key(a, 1, shv, shs);
    const float ws = (a.weight_mode == WM_UNIFORM) ? a.w0 : 1.f;
    const int cls = (ws * sqrtf(vk0) >= ws * sqrtf(vk1)) ? 0 : 1;
    const float vkey = (cls == 0) ? vk0 : vk1;
    if (blockIdx.x == 0 && tid == 0) *a.cls_buf = cls;

    // this CTA's pair and delay chunk in the winning class
    const int npairs = (cls == 0) ? M : M * (M - 1);
    const int cpp = a.cpp_cls[cls], rows = a.rows_cls[cls];
    const int pi = blockIdx.x / cpp, chunk = blockIdx.x - pi * cpp;
    int m = 0, l = 0;
    if (pi < npairs) class_pair(cls, pi, M, m, l);
    const int d_begin = chunk * rows;
    const int d_end = min(a.D, d_begin + rows);
    const int k_first = a.k_lo + d_begin;
    C* out_x = a.part + (size_t)blockIdx.x * 2 * N;
    C* out_h = out_x + N;
    const C zero = make_float2(0.f, 0.f);
    if (pi >= npairs || d_begin >= d_end || !(vkey > 0.f)) {
        for (int i = tid; i < N; i += NT) { out_x[i] = zero; out_h[i] = zero; }
        return;
    }
    // g = eps w (w|chi|/V)^(p-1) chi/|chi|.  With r = key/vkey = (w|chi|/V)^2
    // and sqrt(r) = w_or_1 |chi| / sqrt(vkey) this is
    //     g = eps w_eff r^(p/2 - 1) chi / sqrt(vkey)
    // (w_eff = w for uniform weights, whose key omits w^2; w^2 for a map): no
    // division by |chi|.  p = 8 and 16 take r^3 and r^7 by multiplications,
    // other p the hardware's base-2 exponential and logarithm.
    const float inv_vkey = 1.f / vkey;
    const float inv_vk = rsqrtf(vkey);
    const float expo = a.half_p - 1.f;
    const int pkind = (a.half_p == 4.f) ? 4 : (a.half_p == 8.f) ? 8 : 0;
    const float eps = (float)a.eps;

    for (int n = tid; n < XS; n += NT) xs[n] = (n < N) ? cmul(a.x[(size_t)m * N + n], a.pre[n]) : zero;
    for (int i = tid; i < HS; i += NT) {
        const int p = k_first + i;
        hs[i] = (p >= 0 && p < N) ? a.h[(size_t)l * N + p] : zero;
    }
    for (int i = tid; i < RS * N * (NF > 1 ? 2 : 1); i += NT) ghs[i] = zero;
    __syncthreads();

    const int slot = tid / TPR;
    const int t = tid - slot * TPR;
    C* buf = bufs + slot * PL::padlen;
    C* gh_slot = ghs + slot * N;
    C* gx_slot = gxs + slot * N;
    C gxr[E];                                 // grad x at n = t + TPR q (rows of L >= N bins)
#pragma unroll
    for (int q = 0; q < E; ++q) gxr[q] = zero;

    for (int d0 = d_begin; d0 < d_end; d0 += RS) {
        const int d = d0 + slot;
        const bool row_in = d < d_end;
        const int k = row_in ? a.k_lo + d : k_first;   // rows past the chunk compute on valid data, unused
        const bool live = row_in && !(m == l && k == 0);
        // ---- recompute chi(k, .) exactly as the forward pass does ----
        C v[E];
        const C* xk = xs + t;
        const C* hk = hs + (k - k_first) + t;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            C q = zero;
            for (int c = 0; c < NF; ++c) q = cadd(q, cmulc(xk[r * TPR + c * L], hk[r * TPR + c * L]));
            v[r] = q;
        }
        // The two transforms run through one copy of the FFT code (its size is
        // what the SM's instruction cache sees): chi, then conj(g) -> G2.
#pragma unroll 1
        for (int tr = 0; tr < 2; ++tr) {
        pass_compute<L, E, E, 1>(v, t, tws);
        fft_rest<L, E, 1>(v, t, slot, buf, tws);
        if (tr == 1) break;
        // ---- g per bin, conjugated, into the input layout of the next FFT ----
        // bin of v[s*RL + r] is t + TPR*(s + r*NBL); the next pass 0 reads bin t + TPR*q as v2[q]
        C v2[E];
        const float* wrow = (row_in && a.weight_mode != WM_UNIFORM) ? a.wmap + (size_t)d * L + t : nullptr;
        // one copy of the cell loop per power kind (a uniform branch, no per-cell branch)
        auto form_g = [&](auto kind) {
            constexpr int K = decltype(kind)::value;
#pragma unroll
            for (int r = 0; r < RL; ++r) {
#pragma unroll
                for (int s = 0; s < NBL; ++s) {
                    const int q = s + r * NBL;
                    const C c = v[s * RL + r];
                    const float mag2 = c.x * c.x + c.y * c.y;
                    float w = ws;
                    if (wrow != nullptr) w = __ldg(wrow + TPR * q);
                    const bool map = (wrow != nullptr && a.weight_mode == WM_MAP);
                    const float rr = (map ? w * w * mag2 : mag2) * inv_vkey;
                    float pw;
                    if constexpr (K == 4) {
                        pw = rr * rr * rr;
                    } else if constexpr (K == 8) {
                        const float r2 = rr * rr;
                        pw = r2 * r2 * r2 * rr;
                    } else {
                        pw = ex2_approx(expo * __log2f(rr));
                    }
                    const float coef = (live && w > 0.f && mag2 > 0.f) ? eps * (map ? w * w : w) * pw * inv_vk : 0.f;
                    v2[q] = make_float2(coef * c.x, -coef * c.y);   // conj(g)
                }
            }
        };
        if (pkind == 4) form_g(std::integral_constant<int, 4>{});
        else if (pkind == 8) form_g(std::integral_constant<int, 8>{});
        else form_g(std::integral_constant<int, 0>{});
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = v2[q];
        }
        // ---- accumulate: G2(n) = v[s*RL + r] at n = t + TPR*q (+ c L) ----
        if (live) {
#pragma unroll
            for (int r = 0; r < RL; ++r) {
#pragma unroll
                for (int s = 0; s < NBL; ++s) {
                    const int q = s + r * NBL;
                    const C gt = v[s * RL + r];
                    if (NF == 1) {
                        const int n = t + TPR * q;
                        // h_l(n+k) from the window (zero outside [0, N)); conj(G2) h, added
                        // into the accumulators by fused multiply-adds
                        gxr[q] = cmac_conj(gxr[q], gt, hk[TPR * q]);
                        const int p = n + k;
                        if (p >= 0 && p < N) gh_slot[p] = cmac(gh_slot[p], gt, xk[TPR * q]);
                    } else {
                        for (int c = 0; c < NF; ++c) {
                            const int n = t + TPR * q + c * L;
                            if (n >= N) break;
                            gx_slot[n] = cadd(gx_slot[n], cmul(cconj(gt), hk[TPR * q + c * L]));
                            const int p = n + k;
                            if (p >= 0 && p < N) gh_slot[p] = cadd(gh_slot[p], cmul(gt, xk[TPR * q + c * L]));
                        }
                    }
                }
            }
        }
        row_sync<TPR>(slot);
    }
    __syncthreads();
    // the register partials of grad x go through the (now free) row buffers
    if (NF == 1) {
#pragma unroll
        for (int q = 0; q < E; ++q) bufs[slot * L + t + TPR * q] = gxr[q];
        __syncthreads();
    }
    // ---- fixed-order sum over row slots; grad x takes its phase e^{-j 2 pi nu0 n} here ----
    for (int i = tid; i < N; i += NT) {
        C sx = zero, sh = zero;
        for (int r = 0; r < RS; ++r) {
            sx = cadd(sx, NF == 1 ? bufs[r * L + i] : gxs[r * N + i]);
            sh = cadd(sh, ghs[r * N + i]);
        }
        out_x[i] = cmulc(sx, a.pre[i]);
        out_h[i] = sh;
    }
}

// grad x_r(n) = sum over the winning class's pairs (r, l) and their chunks;
// grad h_r(n) over its pairs (m, r).
__global__ void adj_reduce_kernel(const AdjArgs a) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y, which = blockIdx.z;
    pdl_wait();
    pdl_trigger();
    if (n >= a.N) return;
    const int cls = __ldcg(a.cls_buf);
    const int npairs = (cls == 0) ? a.M : a.M * (a.M - 1);
    const int cpp = a.cpp_cls[cls];
    float2 acc = make_float2(0.f, 0.f);
    for (int pi = 0; pi < npairs; ++pi) {
        int m, l;
        class_pair(cls, pi, a.M, m, l);
        if ((which == 0 ? m : l) != r) continue;
        for (int c = 0; c < cpp; ++c) {
            const size_t cta = (size_t)pi * cpp + c;
            acc = cadd(acc, a.part[cta * 2 * a.N + (size_t)which * a.N + n]);
        }
    }
    a.dense[(size_t)which * a.M * a.N + (size_t)r * a.N + n] = acc;
}

template <int L, int E, int NT>
static int adj_smem(int N, int rpc) {
    return (int)sizeof(float2) * adj_smem_entries<L, E, NT>(N, rpc);
}

template <int L, int E, int NT>
static cudaError_t adj_launch_LE(const AdjArgs& a, cudaStream_t s, bool prepare_only) {
    const int smem = adj_smem<L, E, NT>(a.N, a.rpc_max);
    auto kern = adj_fft_kernel<L, E, NT>;
    cudaError_t e = set_smem_once(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess || prepare_only) return e;
    e = launch_ex(kern, dim3(a.grid), dim3(NT), smem, s, a.pdl != 0, a);
    if (e != cudaSuccess) return e;
    const dim3 rg((a.N + 255) / 256, a.M, 2);
    return launch_ex(adj_reduce_kernel, rg, dim3(256), 0, s, a.pdl != 0, a);
}

// Built shapes X(L, E, NT): 8 or 16 values per thread (the forward pass's
// twiddle tables are shared), 512-thread CTAs for rows of >= 1024 bins.
#define AF_ADJ_SHAPES(X)                                                                                     \
    X(32, 8, 256) X(32, 16, 256) X(64, 8, 256) X(64, 16, 256) X(128, 8, 256) X(128, 16, 256) X(256, 8, 256)  \
    X(256, 16, 256) X(512, 8, 256) X(512, 16, 256) X(1024, 8, 256) X(1024, 16, 256) X(2048, 8, 256)         \
    X(2048, 16, 256) X(4096, 16, 256) X(1024, 16, 512) X(2048, 16, 512) X(4096, 16, 512)

static cudaError_t adj_any(const AdjArgs& a, cudaStream_t s, bool prepare_only) {
    const int NT = a.nt ? a.nt : 256;
#define AF_ADJ_CASE(LL, EE, TT) \
    if (a.L == LL && a.fft_e == EE && NT == TT) return adj_launch_LE<LL, EE, TT>(a, s, prepare_only);
    AF_ADJ_SHAPES(AF_ADJ_CASE)
#undef AF_ADJ_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_adj(const AdjArgs& a, cudaStream_t s) { return adj_any(a, s, false); }

cudaError_t adj_prepare(int L, int N, int E, int NT, int rpc) {
    AdjArgs a{};
    a.L = L; a.N = N; a.fft_e = E; a.nt = NT; a.rpc_max = rpc;
    return adj_any(a, nullptr, true);
}

int adj_smem_bytes(int L, int N, int E, int NT, int rpc) {
#define AF_ADJ_SMEM(LL, EE, TT) \
    if (L == LL && E == EE && NT == TT) return adj_smem<LL, EE, TT>(N, rpc);
    AF_ADJ_SHAPES(AF_ADJ_SMEM)
#undef AF_ADJ_SMEM
    return -1;
}

int adj_threads(int L, int E) { return (L >= 1024 && E == 16) ? 512 : 256; }

// Grid of the adjoint: G = k M (M - 1) CTAs (k M for one waveform), so that
// the M auto pairs take k (M - 1) chunks each and the M (M - 1) cross pairs k
// each; chunks hold a multiple of the row slots.  k minimises the time of the
// class with the longer chunks, waves x (row steps + 1/2), with `slots`
// resident CTAs on the GPU.
void adj_geometry(int M, int D, int L, int E, int NT, int slots, AdjGeom* g) {
    const int RS = NT / (L / E);
    const int Pc = M * (M - 1);
    auto round_rs = [&](int v) { return ((v + RS - 1) / RS) * RS; };
    double best = 1e300;
    *g = AdjGeom{};
    for (int k = 1; k <= 64 * slots && k <= D; ++k) {
        const int G = (M >= 2) ? k * Pc : k;
        const int cpp_a = (M >= 2) ? k * (M - 1) : k, cpp_c = k;
        const int rows_a = round_rs((D + cpp_a - 1) / cpp_a);
        const int rows_c = round_rs((D + cpp_c - 1) / cpp_c);
        const int waves = (G + slots - 1) / slots;
        const int longest = (M >= 2) ? rows_c : rows_a;
        const double cost = (double)waves * ((double)longest / RS + 0.5);
        if (cost < best) {
            best = cost;
            g->grid = G;
            g->cpp[0] = cpp_a; g->cpp[1] = cpp_c;
            g->rows[0] = rows_a; g->rows[1] = (M >= 2) ? rows_c : rows_a;
            g->rpc_max = (M >= 2) ? (rows_a > rows_c ? rows_a : rows_c) : rows_a;
        }
        if (G >= 16 * slots) break;
    }
}

}  // namespace af
