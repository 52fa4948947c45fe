// af_fin.cu -- loss assembly, sparse adjoint, Adam and projection of one
// evaluation, spread over M x ceil(N/128) CTAs (one element per thread).
//
// Every CTA merges the per-CTA sidelobe partials of the forward pass into
// WAPSL/WCPSL (Eqs. 8-9), L_WPSL (Eq. 37), p_m (Eq. 38), L_SNRL (Eq. 41) and
// L (Eq. 42) -- the same merge in the same order, so all CTAs agree -- then
// forms its strip of row m of the gradient.  The exact max is differentiated
// at its winning cell (k*, nu*) of pair (m*, l*), whose complex value chi*
// the forward pass handed over:
//     grad x_m*(n) += g h_l*(n+k*) e^{-j 2 pi nu* n}
//     grad h_l*(p) += conj(g) x_m*(p-k*) e^{+j 2 pi nu* (p-k*)},  g = eps w chi*/|chi*|
// plus the SNRL term at (m, m, 0, 0) and, in the p-norm variant, the dense
// partial gradients of the adjoint kernel.  The chain to the logits is
// dL/du = 2 pi Im(conj(x) grad x) Q_A'(z) z(1-z).  In the optimiser modes the
// CTA applies Adam to its strip; for the filters the projection of Eq. 32
// needs the whole row's norm, so each CTA publishes an FP64 partial norm and
// the last CTA of the row to arrive (atomic counter, no waiting) sums the
// partials in a fixed order and rescales the row.  A CTA reads other
// elements of a row only in modes that write nothing.
//
// Programmatic launch: the kernel may start while the forward pass is still
// running.  Before pdl_wait() it only reads its own element's inputs, which
// the forward pass does not write; every global write comes after it.
#include <math.h>

#include "af_common.cuh"
#include "af_device.cuh"
#include "af_kernels.h"
#include "af_step.cuh"

namespace af {

constexpr int kFT = 128;   // threads per CTA = elements per strip

__device__ __forceinline__ float2 cell_phasor(const FinArgs& a, int j, int n) {
    if (a.grid_fft) return cmul(a.pre[n], a.wL[(j * n) & (a.L - 1)]);
    return a.E[(size_t)n * a.L + j];
}

// sqrt of a non-negative double: FP32 square root refined by one Newton step
// (relative error ~1e-15), avoiding the long FP64 square-root sequence.
__device__ __forceinline__ double sqrt_d(double v) {
    if (!(v > 0.0)) return 0.0;
    const float s = sqrtf((float)v);
    const double r = (double)s;
    return r + (double)((float)fma(-r, r, v) / (2.f * s));
}

__global__ void __launch_bounds__(kFT) fin_kernel(const FinArgs a) {
    const int m = blockIdx.y;
    const int strip = blockIdx.x;
    const int S = gridDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int M = a.M, N = a.N;
    const int n = strip * kFT + tid;
    const bool in = n < N;
    const size_t e = (size_t)m * N + n;

    __shared__ double shd[kFT / 32];
    __shared__ float sk[2][kFT / 32];
    __shared__ long long si[2][kFT / 32];
    __shared__ float2 sc2[2][kFT / 32];
    __shared__ float spv[2][kFT / 32], sps[2][kFT / 32];
    __shared__ double s_terms[8];
    __shared__ double s_pmin2;
    __shared__ float2 s_g;           // sparse coefficient g
    __shared__ int s_cell[4];        // m*, l*, k*, j*  (m* = -1: no sparse term)
    __shared__ float2 s_G;           // SNRL coefficient of row m
    __shared__ float s_adam[2];
    __shared__ int s_ok, s_last;
    __shared__ float s_scale;

    pdl_trigger();

    // ---- 0. this element's inputs (not written by the forward pass) ----------
    const float2 zero2 = make_float2(0.f, 0.f);
    float2 xm = zero2, hm = zero2, mh = zero2, vh = zero2;
    float uu = 0.f, mu = 0.f, vu = 0.f, dy = 0.f;
    if (in) {
        xm = a.x[e];
        hm = a.h_in[e];
        if (a.mode == FIN_ADAM_H) { mh = a.m_h[e]; vh = a.v_h[e]; if (a.snap_best) uu = a.u[e]; }
        if (a.mode == FIN_ADAM_U) { uu = a.u[e]; mu = a.m_u[e]; vu = a.v_u[e]; dy = a.dydz[e]; }
        if (a.mode == FIN_GRAD_U && a.grad_u != nullptr) { uu = a.u[e]; dy = a.dydz[e]; }
    }
    pdl_wait();

    // ---- 1. merge the forward partials per class ------------------------------
    float kb[2] = {-1.f, -1.f};
    long long ib[2] = {0x7fffffffffffffffLL, 0x7fffffffffffffffLL};
    float2 cb[2] = {zero2, zero2};
    float pv[2] = {0.f, 0.f}, ps[2] = {0.f, 0.f};
    constexpr int U = 4;   // partials loaded per thread before any is compared
    for (int b0 = 0; b0 < a.nblk; b0 += U * kFT) {
        long long ids[U];
        float ks[U], vv[U], ss[U];
        float2 cs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = b0 + u * kFT + tid;
            const bool ok = b < a.nblk;
            ids[u] = ok ? a.pidx[b] : -1;
            ks[u] = ok ? a.pkey[b] : -1.f;
            cs[u] = ok ? a.pchi[b] : zero2;
            vv[u] = (ok && a.half_p > 0.f) ? a.pvmax[b] : 0.f;
            ss[u] = (ok && a.half_p > 0.f) ? a.psum[b] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (ids[u] < 0) continue;
            const int pair = (b0 + u * kFT + tid) / a.ctas_per_pair;
            const int cls = (pair / M == pair % M) ? 0 : 1;
            if (fbetter(ks[u], ids[u], kb[cls], ib[cls])) { kb[cls] = ks[u]; ib[cls] = ids[u]; cb[cls] = cs[u]; }
            if (a.half_p > 0.f) pmerge(a.half_p, pv[cls], ps[cls], vv[u], ss[u]);
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            const float ok = __shfl_xor_sync(0xffffffffu, kb[c], o);
            const long long oi = __shfl_xor_sync(0xffffffffu, ib[c], o);
            const float ocx = __shfl_xor_sync(0xffffffffu, cb[c].x, o);
            const float ocy = __shfl_xor_sync(0xffffffffu, cb[c].y, o);
            if (fbetter(ok, oi, kb[c], ib[c])) { kb[c] = ok; ib[c] = oi; cb[c] = make_float2(ocx, ocy); }
            const float ov = __shfl_xor_sync(0xffffffffu, pv[c], o);
            const float os = __shfl_xor_sync(0xffffffffu, ps[c], o);
            if (a.half_p > 0.f) pmerge(a.half_p, pv[c], ps[c], ov, os);
        }
        if (lane == 0) {
            sk[c][tid >> 5] = kb[c]; si[c][tid >> 5] = ib[c]; sc2[c][tid >> 5] = cb[c];
            spv[c][tid >> 5] = pv[c]; sps[c][tid >> 5] = ps[c];
        }
    }

    // ---- 2. SNRL term, one waveform per lane of warp 0 (FP64) -----------------
    if (tid < 32) {
        double p = 0.0, c2 = 0.0;
        double2 cm = make_double2(0.0, 0.0);
        if (lane < M) {
            cm = a.cdiag[lane];
            c2 = cm.x * cm.x + cm.y * cm.y;
            p = sqrt_d(c2) * a.inv_N;                      // p_m = |A_mm(0,0)| / N (Eq. 38)
        }
        const double dev = p - a.ptar;
        double ls = (lane < M) ? dev * dev : 0.0;
        double pmin2 = (lane < M) ? c2 * a.inv_N * a.inv_N : 1e300;
        for (int o = 16; o > 0; o >>= 1) {
            ls += __shfl_xor_sync(0xffffffffu, ls, o);
            pmin2 = fmin(pmin2, __shfl_xor_sync(0xffffffffu, pmin2, o));
        }
        if (lane == m) {
            // G_m = (1-eps)(2/M)(p_m - p_tar)/N * c_m/|c_m|
            const float mag = (float)(p * (double)N);
            const float coef = (mag > 0.f) ? (float)((1.0 - a.eps) * (2.0 / M) * dev * a.inv_N) / mag : 0.f;
            s_G = make_float2(coef * (float)cm.x, coef * (float)cm.y);
        }
        if (lane == 0) {
            s_terms[4] = ls / (double)M;                   // L_SNRL (Eq. 41)
            s_pmin2 = pmin2;
        }
        if (m == 0 && strip == 0 && a.terms != nullptr && lane < M) a.terms[8 + lane] = p;
    }
    __syncthreads();

    // ---- 3. class values, loss, winning cell ---------------------------------
    if (tid == 0) {
        double cv[2];
        long long cell[2];
        float2 chi[2];
        for (int c = 0; c < 2; ++c) {
            float k = sk[c][0];
            long long i = si[c][0];
            float2 x = sc2[c][0];
            float v = spv[c][0], s = sps[c][0];
            for (int w = 1; w < kFT / 32; ++w) {
                if (fbetter(sk[c][w], si[c][w], k, i)) { k = sk[c][w]; i = si[c][w]; x = sc2[c][w]; }
                if (a.half_p > 0.f) pmerge(a.half_p, v, s, spv[c][w], sps[c][w]);
            }
            const double wscale = (a.weight_mode == WM_UNIFORM) ? (double)a.w0 : 1.0;
            const bool any = (k >= 0.f) && (i != 0x7fffffffffffffffLL);
            cell[c] = any ? i : -1;
            chi[c] = x;
            if (!any) cv[c] = 0.0;
            else if (a.half_p > 0.f) cv[c] = wscale * (double)(sqrtf(v) * powf(s, 0.5f / a.half_p));
            else cv[c] = wscale * (double)sqrtf(k);
        }
        const int cls = (cv[0] >= cv[1]) ? 0 : 1;
        const double lw = cv[cls];
        const double ls = s_terms[4];
        s_terms[0] = a.eps * lw + (1.0 - a.eps) * ls;      // Eq. 42
        s_terms[1] = lw; s_terms[2] = cv[0]; s_terms[3] = cv[1];
        s_terms[5] = (double)cls; s_terms[6] = (double)cell[0]; s_terms[7] = (double)cell[1];
        // winning cell of the exact max and its coefficient g = eps w chi/|chi|
        s_cell[0] = -1;
        s_g = zero2;
        if (a.half_p <= 0.f && cell[cls] >= 0) {
            const long long cc = cell[cls];
            int j, d, pair;
            if (cc < 0x7fffffffLL) {
                const unsigned c32 = (unsigned)cc, L32 = (unsigned)a.L, D32 = (unsigned)a.D;
                const unsigned row = c32 / L32;
                j = (int)(c32 - row * L32);
                pair = (int)(row / D32);
                d = (int)(row - (unsigned)pair * D32);
            } else {
                j = (int)(cc % a.L);
                d = (int)((cc / a.L) % a.D);
                pair = (int)(cc / ((long long)a.L * a.D));
            }
            s_cell[0] = pair / M; s_cell[1] = pair % M; s_cell[2] = a.k_lo + d; s_cell[3] = j;
            const float cr = chi[cls].x, ci = chi[cls].y;
            const float mag = sqrtf(cr * cr + ci * ci);
            const float w = (a.weight_mode == WM_UNIFORM) ? a.w0 : a.wmap[(size_t)d * a.L + j];
            if (mag > 0.f) {
                const float f = (float)a.eps * w / mag;
                s_g = make_float2(f * cr, f * ci);
            }
        }
        if (m == 0 && strip == 0) {
            if (a.terms) for (int i = 0; i < 8; ++i) a.terms[i] = s_terms[i];
            if (a.log) {
                const long long o = a.ctr ? a.ctr[0] - 1 : 0;
                double* lg = a.log + ((size_t)o * a.evals_per_outer + a.eval_index) * 4;
                lg[0] = s_terms[0]; lg[1] = s_terms[1]; lg[2] = s_terms[4]; lg[3] = s_terms[5];
            }
            if (!isfinite(s_terms[0]) && a.err_flag) atomicOr(a.err_flag, 1);
        }
    }
    __syncthreads();

    const bool need_gx = (a.mode != FIN_ADAM_H);
    const bool need_gh = (a.mode != FIN_ADAM_U);
    const int ms = s_cell[0], ls_ = s_cell[1], ks = s_cell[2], js = s_cell[3];
    const float2 g = s_g, Gm = s_G;

    // ---- 4. this thread's element of row m of the gradient ---------------------
    float2 gx = zero2, gh = zero2;
    if (in) {
        if (need_gx) {
            gx = cmul(Gm, hm);
            if (m == ms) {
                const int p = n + ks;
                if (p >= 0 && p < N) gx = cadd(gx, cmul(g, cmulc(a.h_in[(size_t)ls_ * N + p], cell_phasor(a, js, n))));
            }
        }
        if (need_gh) {
            gh = cmul(cconj(Gm), xm);
            if (m == ls_ && ms >= 0) {
                const int q = n - ks;
                if (q >= 0 && q < N) gh = cadd(gh, cmul(cconj(g), cmul(a.x[(size_t)ms * N + q], cell_phasor(a, js, q))));
            }
        }
        if (a.dense_g != nullptr) {
            for (int b = 0; b < a.n_dense; ++b) {
                const float2* base = a.dense_g + (size_t)b * 2 * M * N;
                if (need_gx) gx = cadd(gx, base[e]);
                if (need_gh) gh = cadd(gh, base[(size_t)M * N + e]);
            }
        }
    }

    // ---- 5. outputs ---------------------------------------------------------------
    if (a.mode == FIN_GRAD_XH || a.mode == FIN_GRAD_U) {
        if (!in) return;
        bool bad = !isfinite(gx.x) || !isfinite(gx.y) || !isfinite(gh.x) || !isfinite(gh.y);
        if (a.grad_x) a.grad_x[e] = gx;
        if (a.grad_h) a.grad_h[e] = gh;
        if (a.mode == FIN_GRAD_U && a.grad_u != nullptr) {
            const float gy = 6.283185307179586f * (xm.x * gx.y - xm.y * gx.x);
            const float z = sigmoidf_(uu);
            const float gu = gy * dy * z * (1.f - z);
            a.grad_u[e] = gu;
            bad |= !isfinite(gu);
        }
        if (bad && a.err_flag) atomicOr(a.err_flag, 1);
        return;
    }

    // optimiser modes: Adam step counter and bias corrections
    const long long o = a.ctr[0] - 1;
    if (tid == 0) {
        const long long t = (a.mode == FIN_ADAM_H) ? a.ctr[1] + o * a.n_h + a.inner + 1
                                                   : a.ctr[2] + o * a.n_x + a.inner + 1;
        // 1 - beta^t = -expm1(t ln beta), FP32 (relative error ~1e-6 at any t)
        s_adam[0] = -expm1f((float)t * log1pf(a.b1 - 1.f));
        s_adam[1] = -expm1f((float)t * log1pf(a.b2 - 1.f));
        if (a.mode == FIN_ADAM_H && a.snap_best) {
            // best-design record: this evaluation scored the hard design (X_hard, H)
            const double* prev = a.best2 + ((o + 1) & 1) * 4;
            double* cur = a.best2 + (o & 1) * 4;
            // SNRL_m = -20 log10 p_m <= target + 0.05 dB  <=>  p_m^2 >= p_accept2
            s_ok = (s_pmin2 >= a.p_accept2 && s_terms[1] < prev[0]) ? 1 : 0;
            if (m == 0 && strip == 0) {
                if (s_ok) {
                    cur[0] = s_terms[1]; cur[1] = s_terms[0];
                    cur[2] = (double)(a.ctr[3] + o); cur[3] = -10.0 * log10(s_pmin2);
                } else {
                    for (int i = 0; i < 4; ++i) cur[i] = prev[i];
                }
            }
        }
    }
    __syncthreads();
    const float c1 = s_adam[0], c2 = s_adam[1];
    bool bad = false;

    if (a.mode == FIN_ADAM_H) {
        if (a.snap_best && s_ok && in) {
            if (a.best_h) a.best_h[e] = hm;
            if (a.best_q) a.best_q[e] = hard_q(a.qa, sigmoidf_(uu));
        }
        // Adam on (H_Re, H_Im) of this element, then the projection of Eq. 32
        double e2 = 0.0;
        if (in) {
            float2 mm_ = mh, vv = vh, hv = hm;
            mm_.x = a.b1 * mm_.x + (1.f - a.b1) * gh.x;
            mm_.y = a.b1 * mm_.y + (1.f - a.b1) * gh.y;
            vv.x = a.b2 * vv.x + (1.f - a.b2) * gh.x * gh.x;
            vv.y = a.b2 * vv.y + (1.f - a.b2) * gh.y * gh.y;
            hv.x -= a.lr * (mm_.x / c1) / (sqrtf(vv.x / c2) + a.adam_eps);
            hv.y -= a.lr * (mm_.y / c1) / (sqrtf(vv.y / c2) + a.adam_eps);
            a.m_h[e] = mm_;
            a.v_h[e] = vv;
            a.h[e] = hv;                       // unprojected until the row's last CTA rescales it
            e2 = (double)hv.x * hv.x + (double)hv.y * hv.y;
            bad |= !isfinite(hv.x) || !isfinite(hv.y);
        }
        __threadfence();
        e2 = block_sum_d(e2, shd);
        if (tid == 0) {
            a.norm_part[(size_t)m * S + strip] = e2;
            __threadfence();
            const unsigned prev_arrivals = atomicAdd(a.row_ctr + m, 1u);
            s_last = (prev_arrivals == (unsigned)(S - 1)) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (tid == 0) {
                double tot = 0.0;
                for (int s = 0; s < S; ++s) tot += __ldcg(a.norm_part + (size_t)m * S + s);
                s_scale = (tot > 0.0) ? (float)sqrt_d((double)N / tot) : 1.f;
                a.row_ctr[m] = 0u;
                if (!isfinite(s_scale) && a.err_flag) atomicOr(a.err_flag, 1);
            }
            __syncthreads();
            const float sc = s_scale;
            for (int i = tid; i < N; i += kFT) {
                float2* hp = a.h + (size_t)m * N + i;
                const float2 v = __ldcg(hp);
                *hp = make_float2(v.x * sc, v.y * sc);
            }
        }
    } else if (in) {  // FIN_ADAM_U
        const float gy = 6.283185307179586f * (xm.x * gx.y - xm.y * gx.x);
        const float z = sigmoidf_(uu);
        const float gg = gy * dy * z * (1.f - z);
        const float mm_ = a.b1 * mu + (1.f - a.b1) * gg;
        const float vv = a.b2 * vu + (1.f - a.b2) * gg * gg;
        uu -= a.lr * (mm_ / c1) / (sqrtf(vv / c2) + a.adam_eps);
        a.m_u[e] = mm_;
        a.v_u[e] = vv;
        a.u[e] = uu;
        bad |= !isfinite(uu);
    }
    if (bad && a.err_flag) atomicOr(a.err_flag, 1);

    // waveform of the next evaluation (this element only; depends on u alone)
    if (a.next_wave != NEXT_NONE && in) {
        const float z = sigmoidf_((a.mode == FIN_ADAM_U) ? uu : a.u[e]);
        if (a.next_wave == NEXT_HARD) {
            a.x_next[e] = a.qa.level[hard_q(a.qa, z) % a.qa.B];
        } else {
            float2 xv;
            float d;
            soft_q(a.qa, z, nullptr, &d, &xv);
            a.x_next[e] = xv;
            a.dydz_next[e] = d;
        }
    }
}

int fin_strips(int N) { return (N + kFT - 1) / kFT; }

cudaError_t launch_fin(const FinArgs& a, cudaStream_t s) {
    const dim3 grid(fin_strips(a.N), a.M);
    return launch_ex(fin_kernel, grid, dim3(kFT), 0, s, a.pdl != 0, a);
}

}  // namespace af
