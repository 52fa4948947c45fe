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

namespace af {

constexpr int kFinThreads = 256;
constexpr int kMaxPerThread = 16;   // N <= 4096 = 16 * 256

__device__ __forceinline__ float sigmoidf_(float u) { return 1.f / (1.f + expf(-u)); }

__device__ __forceinline__ int lower_bound_f(const float* v, int n, float x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (v[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int upper_bound_f(const float* v, int n, float x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (v[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Number of thresholds <= v (upper bound).  For the uniform set
// rho_i = (i + 1/2)/K the answer is within one of floor(K v + 1/2); the table
// is then consulted at most twice, so the count is exact for any v.
__device__ __forceinline__ int count_le(const QuantArgs& q, float v) {
    if (!q.uniform) return upper_bound_f(q.rho, q.K, v);
    int c = (int)floorf(fminf(fmaxf(v, -1.f), 2.f) * (float)q.K + 0.5f);
    c = min(max(c, 0), q.K);
    if (c > 0 && __ldg(q.rho + c - 1) > v) --c;
    else if (c < q.K && __ldg(q.rho + c) <= v) ++c;
    return c;
}
// Number of thresholds < v (lower bound), same scheme.
__device__ __forceinline__ int count_lt(const QuantArgs& q, float v) {
    if (!q.uniform) return lower_bound_f(q.rho, q.K, v);
    int c = (int)ceilf(fminf(fmaxf(v, -1.f), 2.f) * (float)q.K - 0.5f);
    c = min(max(c, 0), q.K);
    if (c > 0 && __ldg(q.rho + c - 1) >= v) --c;
    else if (c < q.K && __ldg(q.rho + c) < v) ++c;
    return c;
}

// Soft quantizer of Eq. 24 at z.  Thresholds more than `win` below z have
// tanh = +1 and those more than `win` above have tanh = -1 in FP32, so only
// the window is evaluated; the saturated ones add 2a each = i0 / B.
__device__ __forceinline__ void soft_q(const QuantArgs& q, float z, float* y, float* dydz, float2* x) {
    const int i0 = count_lt(q, z - q.win);
    const int i1 = count_le(q, z + q.win);
    float s = 0.f, ds = 0.f;
    for (int i = i0; i < i1; ++i) {
        const float t = tanhf(q.c * (z - q.rho[i]));
        s += q.a * (t + 1.f);
        ds += q.a * q.c * (1.f - t * t);
    }
    if (y) *y = (float)i0 * (2.f * q.a) + s;
    if (dydz) *dydz = ds;
    if (x) {
        // phase in cycles: i0/B + s, reduced modulo 1 before sincospi
        float f = (float)(i0 % q.B) / (float)q.B + s;
        f -= floorf(f);
        float sn, cs;
        sincospif(2.f * f, &sn, &cs);
        *x = make_float2(cs, sn);
    }
}

__device__ __forceinline__ int hard_q(const QuantArgs& q, float z) { return count_le(q, z); }

// ------------------------------------------------------------ wave kernels --
__global__ void wave_from_logits_kernel(const float* __restrict__ u, int n, QuantArgs q, int hard,
                                        float2* __restrict__ x, float* __restrict__ dydz,
                                        int32_t* __restrict__ qout) {
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

// FP64 hard waveform and FP64 copy of the filters for the acceptance pass.
__global__ void wave_hard_f64_kernel(const float* __restrict__ u, const float2* __restrict__ h, int n,
                                     QuantArgs q, const double2* __restrict__ level64,
                                     double2* __restrict__ x64, double2* __restrict__ h64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int qq = hard_q(q, sigmoidf_(u[i]));
    x64[i] = level64[qq % q.B];
    const float2 hv = h[i];
    h64[i] = make_double2((double)hv.x, (double)hv.y);
}

// ------------------------------------------------------- block reductions --
template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum_d(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;
}

__device__ __forceinline__ bool fbetter(float a, long long ia, float b, long long ib) {
    return a > b || (a == b && ia < ib);
}

__device__ __forceinline__ void pmerge(float hp, float& v, float& s, float ov, float os) {
    if (ov <= 0.f) return;
    if (v <= 0.f) { v = ov; s = os; return; }
    const float nv = fmaxf(v, ov);
    s = s * exp2f(hp * __log2f(v / nv)) + os * exp2f(hp * __log2f(ov / nv));
    v = nv;
}

__device__ __forceinline__ float2 cell_phasor(const FinArgs& a, int j, int n) {
    if (a.grid_fft) return cmul(a.pre[n], a.wL[(j * n) & (a.L - 1)]);
    return a.E[(size_t)n * a.L + j];
}

// ------------------------------------------------------------- fin kernel --
__global__ void __launch_bounds__(kFinThreads) fin_kernel(const FinArgs a) {
    const int m = blockIdx.x;
    const int tid = threadIdx.x;
    const int M = a.M, N = a.N;
    __shared__ double shd[kFinThreads / 32];
    __shared__ float sk[2][kFinThreads / 32];
    __shared__ long long si[2][kFinThreads / 32];
    __shared__ float spv[2][kFinThreads / 32], sps[2][kFinThreads / 32];
    __shared__ double s_terms[8];
    __shared__ double2 s_g;          // sparse coefficient g
    __shared__ int s_cell[4];        // m*, l*, k*, j*  (m* = -1: no sparse term)
    __shared__ float s_adam[3];
    __shared__ float2 s_G;           // SNRL coefficient of this row
    __shared__ float s_scale;        // projection factor
    __shared__ int s_ok;             // best-design decision

    // ---- 1. merge the forward partials per class --------------------------
    float kb[2] = {-1.f, -1.f};
    long long ib[2] = {0x7fffffffffffffffLL, 0x7fffffffffffffffLL};
    float pv[2] = {0.f, 0.f}, ps[2] = {0.f, 0.f};
    for (int b = tid; b < a.nblk; b += kFinThreads) {
        const long long id = a.pidx[b];
        if (id < 0) continue;
        const int pair = b / a.ctas_per_pair;
        const int cls = (pair / M == pair % M) ? 0 : 1;
        const float k = a.pkey[b];
        if (fbetter(k, id, kb[cls], ib[cls])) { kb[cls] = k; ib[cls] = id; }
        if (a.half_p > 0.f) pmerge(a.half_p, pv[cls], ps[cls], a.pvmax[b], a.psum[b]);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            const float ok = __shfl_xor_sync(0xffffffffu, kb[c], o);
            const long long oi = __shfl_xor_sync(0xffffffffu, ib[c], o);
            if (fbetter(ok, oi, kb[c], ib[c])) { kb[c] = ok; ib[c] = oi; }
            const float ov = __shfl_xor_sync(0xffffffffu, pv[c], o);
            const float os = __shfl_xor_sync(0xffffffffu, ps[c], o);
            if (a.half_p > 0.f) pmerge(a.half_p, pv[c], ps[c], ov, os);
        }
        if ((tid & 31) == 0) {
            sk[c][tid >> 5] = kb[c]; si[c][tid >> 5] = ib[c];
            spv[c][tid >> 5] = pv[c]; sps[c][tid >> 5] = ps[c];
        }
    }
    __syncthreads();
    if (tid == 0) {
        double cv[2];
        long long cell[2];
        for (int c = 0; c < 2; ++c) {
            float k = sk[c][0];
            long long i = si[c][0];
            float v = spv[c][0], s = sps[c][0];
            for (int w = 1; w < kFinThreads / 32; ++w) {
                if (fbetter(sk[c][w], si[c][w], k, i)) { k = sk[c][w]; i = si[c][w]; }
                if (a.half_p > 0.f) pmerge(a.half_p, v, s, spv[c][w], sps[c][w]);
            }
            const double wscale = (a.weight_mode == WM_UNIFORM) ? (double)a.w0 : 1.0;
            const bool any = (k >= 0.f) && (i != 0x7fffffffffffffffLL);
            cell[c] = any ? i : -1;
            if (!any) cv[c] = 0.0;
            else if (a.half_p > 0.f) cv[c] = wscale * sqrt((double)v) * pow((double)s, 0.5 / (double)a.half_p);
            else cv[c] = wscale * sqrt((double)k);
        }
        const int cls = (cv[0] >= cv[1]) ? 0 : 1;
        const double lw = cv[cls];
        double ls = 0.0;
        for (int mm = 0; mm < M; ++mm) {
            const double2 c = a.cdiag[mm];
            const double p = sqrt(c.x * c.x + c.y * c.y) / (double)N;
            ls += (p - a.ptar) * (p - a.ptar);
        }
        ls /= (double)M;
        s_terms[0] = a.eps * lw + (1.0 - a.eps) * ls;
        s_terms[1] = lw; s_terms[2] = cv[0]; s_terms[3] = cv[1]; s_terms[4] = ls;
        s_terms[5] = (double)cls; s_terms[6] = (double)cell[0]; s_terms[7] = (double)cell[1];
        // winning cell of the exact max
        s_cell[0] = -1;
        if (a.half_p <= 0.f && cell[cls] >= 0) {
            const long long cc = cell[cls];
            const int j = (int)(cc % a.L);
            const int d = (int)((cc / a.L) % a.D);
            const int pair = (int)(cc / ((long long)a.L * a.D));
            s_cell[0] = pair / M; s_cell[1] = pair % M; s_cell[2] = a.k_lo + d; s_cell[3] = j;
        }
        if (m == 0) {
            if (a.terms) {
                for (int i = 0; i < 8; ++i) a.terms[i] = s_terms[i];
                for (int mm = 0; mm < M; ++mm) {
                    const double2 c = a.cdiag[mm];
                    a.terms[8 + mm] = sqrt(c.x * c.x + c.y * c.y) / (double)N;
                }
            }
            if (a.log) {
                const long long o = a.ctr ? a.ctr[0] - 1 : 0;
                double* lg = a.log + ((size_t)o * a.evals_per_outer + a.eval_index) * 4;
                lg[0] = s_terms[0]; lg[1] = s_terms[1]; lg[2] = s_terms[4]; lg[3] = s_terms[5];
            }
            if (!isfinite(s_terms[0]) && a.err_flag) atomicExch(a.err_flag, 1);
        }
    }
    __syncthreads();

    const bool need_gx = (a.mode != FIN_ADAM_H);
    const bool need_gh = (a.mode != FIN_ADAM_U);
    const int ms = s_cell[0], ls_ = s_cell[1], ks = s_cell[2], js = s_cell[3];

    // ---- 2. chi at the winning cell (only the CTAs that need it) -----------
    if (tid == 0) s_g = make_double2(0.0, 0.0);
    const bool mine = (ms >= 0) && ((need_gx && m == ms) || (need_gh && m == ls_));
    if (mine) {
        double cr = 0.0, ci = 0.0;
        for (int n = tid; n < N; n += kFinThreads) {
            const int p = n + ks;
            if (p < 0 || p >= N) continue;
            const float2 t = cmul(cmulc(a.x[(size_t)ms * N + n], a.h_in[(size_t)ls_ * N + p]), cell_phasor(a, js, n));
            cr += t.x; ci += t.y;
        }
        cr = block_sum_d(cr, shd);
        ci = block_sum_d(ci, shd);
        if (tid == 0) {
            const double mag = sqrt(cr * cr + ci * ci);
            const double w = (a.weight_mode == WM_UNIFORM) ? (double)a.w0
                                                           : (double)a.wmap[(size_t)(ks - a.k_lo) * a.L + js];
            if (mag > 0.0) s_g = make_double2(a.eps * w * cr / mag, a.eps * w * ci / mag);
        }
    }
    // SNRL coefficient G_m = (1-eps)(2/M)(p_m - p_tar)/N * c_m/|c_m| (FP64, once)
    if (tid == 0) {
        const double2 c = a.cdiag[m];
        const double mag = sqrt(c.x * c.x + c.y * c.y);
        s_G = make_float2(0.f, 0.f);
        if (mag > 0.0) {
            const double coef = (1.0 - a.eps) * (2.0 / M) * (mag / N - a.ptar) / N / mag;
            s_G = make_float2((float)(coef * c.x), (float)(coef * c.y));
        }
    }
    __syncthreads();
    const float2 g = make_float2((float)s_g.x, (float)s_g.y);
    const float2 Gm = s_G;

    // ---- 3. row m of the gradient ------------------------------------------
    float2 gx[kMaxPerThread], gh[kMaxPerThread];
    const int nper = (N + kFinThreads - 1) / kFinThreads;
#pragma unroll
    for (int i = 0; i < kMaxPerThread; ++i) {
        const int n = tid + i * kFinThreads;
        float2 vx = make_float2(0.f, 0.f), vh = make_float2(0.f, 0.f);
        if (n < N) {
            const float2 xm = a.x[(size_t)m * N + n];
            const float2 hm = a.h_in[(size_t)m * N + n];
            if (need_gx) {
                vx = cmul(Gm, hm);
                if (m == ms) {
                    const int p = n + ks;
                    if (p >= 0 && p < N)
                        vx = cadd(vx, cmul(g, cmulc(a.h_in[(size_t)ls_ * N + p], cell_phasor(a, js, n))));
                }
            }
            if (need_gh) {
                vh = cmul(cconj(Gm), xm);
                if (m == ls_ && ms >= 0) {
                    const int q = n - ks;
                    if (q >= 0 && q < N)
                        vh = cadd(vh, cmul(cconj(g), cmul(a.x[(size_t)ms * N + q], cell_phasor(a, js, q))));
                }
            }
            if (a.dense_g != nullptr) {
                for (int b = 0; b < a.n_dense; ++b) {
                    const float2* base = a.dense_g + (size_t)b * 2 * M * N;
                    if (need_gx) vx = cadd(vx, base[(size_t)m * N + n]);
                    if (need_gh) vh = cadd(vh, base[(size_t)M * N + (size_t)m * N + n]);
                }
            }
        }
        gx[i] = vx;
        gh[i] = vh;
    }

    // ---- 4. outputs --------------------------------------------------------
    if (a.mode == FIN_GRAD_XH || a.mode == FIN_GRAD_U) {
        bool bad = false;
#pragma unroll
        for (int i = 0; i < kMaxPerThread; ++i) {
            const int n = tid + i * kFinThreads;
            if (i >= nper || n >= N) continue;
            const size_t e = (size_t)m * N + n;
            if (a.grad_x) a.grad_x[e] = gx[i];
            if (a.grad_h) a.grad_h[e] = gh[i];
            if (a.mode == FIN_GRAD_U && a.grad_u != nullptr) {
                const float2 xv = a.x[e];
                const float gy = 6.283185307179586f * (xv.x * gx[i].y - xv.y * gx[i].x);
                const float z = sigmoidf_(a.u[e]);
                const float gu = gy * a.dydz[e] * z * (1.f - z);
                a.grad_u[e] = gu;
                bad |= !isfinite(gu);
            }
            bad |= !isfinite(gx[i].x) || !isfinite(gx[i].y) || !isfinite(gh[i].x) || !isfinite(gh[i].y);
        }
        if (bad && a.err_flag) atomicExch(a.err_flag, 1);
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
    }
    __syncthreads();
    const float c1 = s_adam[0], c2 = s_adam[1];

    if (a.mode == FIN_ADAM_H) {
        // best-design record: this evaluation scored the hard design (X_hard, H)
        if (a.snap_best) {
            const double* prev = a.best2 + ((o + 1) & 1) * 4;
            double* cur = a.best2 + (o & 1) * 4;
            // SNRL_m = -20 log10 p_m <= target + 0.05 dB  <=>  p_m^2 >= p_min^2
            if (tid == 0) {
                double pmin2 = 1e300;
                for (int mm = 0; mm < M; ++mm) {
                    const double2 c = a.cdiag[mm];
                    pmin2 = fmin(pmin2, (c.x * c.x + c.y * c.y) / ((double)N * N));
                }
                s_ok = (pmin2 >= a.p_accept2 && s_terms[1] < prev[0]) ? 1 : 0;
                if (m == 0) {
                    if (s_ok) {
                        cur[0] = s_terms[1]; cur[1] = s_terms[0];
                        cur[2] = (double)(a.ctr[3] + o); cur[3] = -10.0 * log10(pmin2);
                    } else {
                        for (int i = 0; i < 4; ++i) cur[i] = prev[i];
                    }
                }
            }
            __syncthreads();
            const bool ok = s_ok != 0;
            if (ok) {
                for (int i = 0; i < nper; ++i) {
                    const int n = tid + i * kFinThreads;
                    if (n >= N) break;
                    const size_t e = (size_t)m * N + n;
                    if (a.best_h) a.best_h[e] = a.h[e];
                    if (a.best_q) a.best_q[e] = hard_q(a.qa, sigmoidf_(a.u[e]));
                }
            }
        }
        // Adam on (H_Re, H_Im), then the projection of Eq. 32
        float2 hn[kMaxPerThread];
        double e2 = 0.0;
#pragma unroll
        for (int i = 0; i < kMaxPerThread; ++i) {
            const int n = tid + i * kFinThreads;
            if (i >= nper || n >= N) continue;
            const size_t e = (size_t)m * N + n;
            float2 mm_ = a.m_h[e], vv = a.v_h[e], hv = a.h[e];
            const float2 gg = gh[i];
            mm_.x = a.b1 * mm_.x + (1.f - a.b1) * gg.x;
            mm_.y = a.b1 * mm_.y + (1.f - a.b1) * gg.y;
            vv.x = a.b2 * vv.x + (1.f - a.b2) * gg.x * gg.x;
            vv.y = a.b2 * vv.y + (1.f - a.b2) * gg.y * gg.y;
            hv.x -= a.lr * (mm_.x / c1) / (sqrtf(vv.x / c2) + a.adam_eps);
            hv.y -= a.lr * (mm_.y / c1) / (sqrtf(vv.y / c2) + a.adam_eps);
            a.m_h[e] = mm_;
            a.v_h[e] = vv;
            hn[i] = hv;
            e2 += (double)hv.x * hv.x + (double)hv.y * hv.y;
        }
        e2 = block_sum_d(e2, shd);
        if (tid == 0) s_scale = (e2 > 0.0) ? (float)sqrt((double)N / e2) : 1.f;
        __syncthreads();
        const float sc = s_scale;
        bool bad = !isfinite(sc);
#pragma unroll
        for (int i = 0; i < kMaxPerThread; ++i) {
            const int n = tid + i * kFinThreads;
            if (i >= nper || n >= N) continue;
            const size_t e = (size_t)m * N + n;
            a.h[e] = make_float2(hn[i].x * sc, hn[i].y * sc);
            bad |= !isfinite(hn[i].x) || !isfinite(hn[i].y);
        }
        if (bad && a.err_flag) atomicExch(a.err_flag, 1);
    } else {  // FIN_ADAM_U
        bool bad = false;
#pragma unroll
        for (int i = 0; i < kMaxPerThread; ++i) {
            const int n = tid + i * kFinThreads;
            if (i >= nper || n >= N) continue;
            const size_t e = (size_t)m * N + n;
            const float2 xv = a.x[e];
            const float gy = 6.283185307179586f * (xv.x * gx[i].y - xv.y * gx[i].x);
            float uu = a.u[e];
            const float z = sigmoidf_(uu);
            const float gg = gy * a.dydz[e] * z * (1.f - z);
            float mm_ = a.b1 * a.m_u[e] + (1.f - a.b1) * gg;
            float vv = a.b2 * a.v_u[e] + (1.f - a.b2) * gg * gg;
            uu -= a.lr * (mm_ / c1) / (sqrtf(vv / c2) + a.adam_eps);
            a.m_u[e] = mm_;
            a.v_u[e] = vv;
            a.u[e] = uu;
            bad |= !isfinite(uu);
        }
        if (bad && a.err_flag) atomicExch(a.err_flag, 1);
    }
    __syncthreads();

    // waveform of the next evaluation (own row only)
    if (a.next_wave != NEXT_NONE) {
#pragma unroll
        for (int i = 0; i < kMaxPerThread; ++i) {
            const int n = tid + i * kFinThreads;
            if (i >= nper || n >= N) continue;
            const size_t e = (size_t)m * N + n;
            const float z = sigmoidf_(a.u[e]);
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
    wave_from_logits_kernel<<<(n + 255) / 256, 256, 0, s>>>(u, n, q, hard, x, dydz, qout);
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
cudaError_t launch_fin(const FinArgs& a, cudaStream_t s) {
    fin_kernel<<<a.M, kFinThreads, 0, s>>>(a);
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
