// af_device.cuh -- device helpers shared by the per-step kernels: sigmoid,
// threshold counting, the quantizers of Eqs. 24 and 43, block reductions.
#pragma once

#include <math.h>

#include "af_common.cuh"
#include "af_step.cuh"

namespace af {

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

// Threshold i of the uniform set rho_i = (i + 1/2)/K, bit-identical to the
// table the host builds as the FP32 rounding of the FP64 quotient: the exact
// value (2i+1)/(2K) has 2K <= 2^21, so it lies at least 2^-45 (relative)
// away from any FP32 rounding boundary it does not sit on, and it sits on one
// only if it is a dyadic fraction of at most 21 bits (then it is exact).  The
// FP64 rounding therefore cannot move it across a boundary, and the FP32
// division of the exact operands 2i+1 and 2K returns the same float.
__device__ __forceinline__ float rho_uniform(int i, int K) {
    return __fdiv_rn((float)(2 * i + 1), (float)(2 * K));
}

// Number of thresholds <= v (upper bound).  For the uniform set the answer is
// within one of floor(K v + 1/2); one or two thresholds, computed as the table
// holds them, settle it, so the count is exact for any v and reads no memory.
__device__ __forceinline__ int count_le(const QuantArgs& q, float v) {
    if (!q.uniform) return upper_bound_f(q.rho, q.K, v);
    int c = (int)floorf(fminf(fmaxf(v, -1.f), 2.f) * (float)q.K + 0.5f);
    c = min(max(c, 0), q.K);
    if (c > 0 && rho_uniform(c - 1, q.K) > v) --c;
    else if (c < q.K && rho_uniform(c, q.K) <= v) ++c;
    return c;
}
// Number of thresholds < v (lower bound), same scheme.
__device__ __forceinline__ int count_lt(const QuantArgs& q, float v) {
    if (!q.uniform) return lower_bound_f(q.rho, q.K, v);
    int c = (int)ceilf(fminf(fmaxf(v, -1.f), 2.f) * (float)q.K - 0.5f);
    c = min(max(c, 0), q.K);
    if (c > 0 && rho_uniform(c - 1, q.K) >= v) --c;
    else if (c < q.K && rho_uniform(c, q.K) < v) ++c;
    return c;
}

// Soft quantizer of Eq. 24 at z.  Thresholds more than `win` below z have
// tanh = +1 and those more than `win` above have tanh = -1 in FP32 (win =
// 9.5/c: tanh(9.5) rounds to 1), so only the window is evaluated; the
// saturated ones add 2a each = i0 / B.
//
// Uniform thresholds rho_i = (i + 1/2)/K: with e_i = e^{2c(z - rho_i)},
// tanh(c(z - rho_i)) = 1 - 2/(1 + e_i) and 1 - tanh^2 = 4 e_i/(1 + e_i)^2, and
// e_{i+1} = e_i e^{-2c/K}.  The sum is taken outward from the threshold
// nearest z (where tanh is not saturated and the recursion has taken no
// steps), each e_i by one multiply; the terms far from z, where the
// accumulated rounding of the recursion grows, are saturated.
//
// When the tanh width 1/c spans at least four threshold spacings (alpha =
// 2c/K <= 1/2, which holds at K = B r_n = 1600 or 6400 with c = 300) the
// uniform sum has a closed form instead, soft_q_closed below, which costs the
// same at any K.
__device__ __forceinline__ void soft_q_closed(const QuantArgs& q, float z, float* y, float* dydz, float2* x);

__device__ __forceinline__ bool soft_q_closed_ok(const QuantArgs& q) {
    return q.uniform && 4.f * q.c <= (float)q.K;     // alpha = 2c/K <= 1/2
}

__device__ __forceinline__ void soft_q(const QuantArgs& q, float z, float* y, float* dydz, float2* x) {
    if (soft_q_closed_ok(q)) {
        soft_q_closed(q, z, y, dydz, x);
        return;
    }
    int i0, i1;
    if (q.uniform) {
        // The window's edges need no exact count: a threshold misplaced across
        // an edge by rounding is saturated there and adds 2a (below) or 0
        // (above) whichever side counts it, so plain arithmetic does.
        const float kz = fminf(fmaxf(z, -1.f), 2.f) * (float)q.K;
        const float kw = q.win * (float)q.K;
        i0 = min(max((int)ceilf(kz - kw - 0.5f), 0), q.K);
        i1 = min(max((int)floorf(kz + kw + 0.5f), i0), q.K);
    } else {
        i0 = count_lt(q, z - q.win);
        i1 = count_le(q, z + q.win);
    }
    float s = 0.f, ds = 0.f;
    if (q.uniform) {
        if (i1 > i0) {
            const float invK = 1.f / (float)q.K;
            const int ic = min(max((int)floorf(z * (float)q.K), i0), i1 - 1);
            const float c2 = 2.f * q.c;
            const float r_up = expf(-c2 * invK);         // e_{i+1} / e_i
            const float r_dn = expf(c2 * invK);          // e_{i-1} / e_i
            const float r_up2 = r_up * r_up, r_dn2 = r_dn * r_dn;
            // four interleaved chains (two upward from ic, two downward from
            // ic - 1), each stepping two thresholds, so the in-order pipeline
            // always has independent work; terms past either end of the window
            // are masked out.  1/(1+e) uses the hardware reciprocal (~1 ulp):
            // e -> inf gives 0 and e -> 0 gives 1, the saturated limits.
            float eu0 = expf(c2 * (z - ((float)ic + 0.5f) * invK));
            float ed0 = expf(c2 * (z - ((float)ic - 0.5f) * invK));
            float eu1 = eu0 * r_up, ed1 = ed0 * r_dn;
            const int n_up = i1 - ic, n_dn = ic - i0;
            const int n_it = max(n_up, n_dn);
            float si0 = 0.f, si1 = 0.f, si2 = 0.f, si3 = 0.f;   // sum 1/(1+e)
            float sd0 = 0.f, sd1 = 0.f, sd2 = 0.f, sd3 = 0.f;   // sum e/(1+e)^2
            for (int t = 0; t < n_it; t += 2) {
                // past its end a downward chain may overflow to inf: selects, not
                // multiplications by 0, keep those terms out
                const float i0_ = __fdividef(1.f, 1.f + eu0), i1_ = __fdividef(1.f, 1.f + eu1);
                const float i2_ = __fdividef(1.f, 1.f + ed0), i3_ = __fdividef(1.f, 1.f + ed1);
                if (t < n_up) { si0 += i0_; sd0 = fmaf(eu0 * i0_, i0_, sd0); }
                if (t + 1 < n_up) { si1 += i1_; sd1 = fmaf(eu1 * i1_, i1_, sd1); }
                if (t < n_dn) { si2 += i2_; sd2 = fmaf(ed0 * i2_, i2_, sd2); }
                if (t + 1 < n_dn) { si3 += i3_; sd3 = fmaf(ed1 * i3_, i3_, sd3); }
                eu0 *= r_up2; eu1 *= r_up2; ed0 *= r_dn2; ed1 *= r_dn2;
            }
            const float sum_inv = (si0 + si1) + (si2 + si3);
            const float sum_d = (sd0 + sd1) + (sd2 + sd3);
            // sum a (tanh + 1) = a (2 W - 2 sum_inv);  sum a c (1 - tanh^2) = 4 a c sum_d
            s = 2.f * q.a * ((float)(i1 - i0) - sum_inv);
            ds = 4.f * q.a * q.c * sum_d;
        }
    } else {
        for (int i = i0; i < i1; ++i) {
            const float t = tanhf(q.c * (z - q.rho[i]));
            s += q.a * (t + 1.f);
            ds += q.a * q.c * (1.f - t * t);
        }
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

// Closed form of Eq. 24 for the uniform thresholds rho_i = (i + 1/2)/K with
// a_i = a.  With tanh(u) + 1 = 2 s(2u) (s the logistic function) the sum is
// y(z) = 2a S(z), S(z) = sum_{i<K} s(alpha (x - i)), alpha = 2c/K, x = zK - 1/2:
// a sum of a smooth function at unit spacing.  The midpoint Euler-Maclaurin
// formula over [-1/2, K - 1/2] turns it into the integral plus end terms:
//   S = zK + [sp(-v0) - sp(v1)]/alpha + (alpha/24)[d1(v1) - d1(v0)]
//         - (7 alpha^3/5760)[d3(v1) - d3(v0)] + R,
// with v0 = 2cz and v1 = 2c(z - 1) the arguments at the two ends, sp the
// softplus log(1 + e^v) (the integral of s), and d1 = s(1 - s), d3 =
// d1 (1 - 6 d1) its first and third derivatives.  The summand is analytic in
// a strip of half-width pi/alpha, so the error of the midpoint rule over the
// whole line is of order e^{-2 pi^2/alpha} (e^{-52} at alpha = 3/8), and the
// next end term is below 1e-7 for alpha <= 1/2: both far below FP32
// resolution.  Its derivative gives Q_A'(z) = 2a dS/dz:
//   dS/dz = K[s(v0) - s(v1)] + 2c (alpha/24)[d2(v1) - d2(v0)]
//         - 2c (7 alpha^3/5760)[d4(v1) - d4(v0)],
// d2 = d1 (1 - 2s) and d4 = d1 (1 - 2s)(1 - 12 d1) the second and fourth
// derivatives.  y = 2aK z + 2a (S - zK): the first product is split exactly
// (hi + lo by a fused multiply-add), so that the phase y mod 1 keeps the
// precision of the small remainder instead of that of y (up to r_n).
__device__ __forceinline__ void soft_q_closed(const QuantArgs& q, float z, float* y, float* dydz, float2* x) {
    const float K = (float)q.K, c = q.c, a2 = 2.f * q.a;
    const float al = 2.f * c / K;
    const float v0 = 2.f * c * z, v1 = 2.f * c * (z - 1.f);
    const float e0 = expf(-fabsf(v0)), e1 = expf(-fabsf(v1));
    const float sp0 = fmaxf(-v0, 0.f) + log1pf(e0);          // sp(-v0)
    const float sp1 = fmaxf(v1, 0.f) + log1pf(e1);           // sp(v1)
    const float r0 = 1.f / (1.f + e0), r1 = 1.f / (1.f + e1);
    const float s0 = (v0 >= 0.f) ? r0 : e0 * r0;             // s(v0)
    const float s1 = (v1 >= 0.f) ? r1 : e1 * r1;             // s(v1)
    const float t0 = e0 * r0 * r0, t1 = e1 * r1 * r1;       // d1(v0), d1(v1): e^{-|v|}/(1 + e^{-|v|})^2
    const float k1 = al * (1.f / 24.f), k3 = al * al * al * (7.f / 5760.f);
    const float rem = (sp0 - sp1) / al + k1 * (t1 - t0) - k3 * (t1 * (1.f - 6.f * t1) - t0 * (1.f - 6.f * t0));
    const float P = a2 * K;
    const float hi = P * z;
    const float r = fmaf(P, z, -hi) + a2 * rem;
    if (y) *y = hi + r;
    if (dydz) {
        const float g0 = t0 * (1.f - 2.f * s0), g1 = t1 * (1.f - 2.f * s1);
        const float dS = K * (s0 - s1) + 2.f * c * (k1 * (g1 - g0) -
                         k3 * (g1 * (1.f - 12.f * t1) - g0 * (1.f - 12.f * t0)));
        *dydz = a2 * dS;
    }
    if (x) {
        float f = (hi - floorf(hi)) + r;
        f -= floorf(f);
        float sn, cs;
        sincospif(2.f * f, &sn, &cs);
        *x = make_float2(cs, sn);
    }
}

__device__ __forceinline__ int hard_q(const QuantArgs& q, float z) { return count_le(q, z); }

// ------------------------------------------------------- block reductions --
template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
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

}  // namespace af
