// af_common.cuh -- complex helpers, register DFTs and shared-memory Stockham
// passes used by the ambiguity-function kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <utility>

namespace af {

// ---------------------------------------------------------------- complex --
template <typename T> struct cx_of;
template <> struct cx_of<float> { using type = float2; };
template <> struct cx_of<double> { using type = double2; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
// acc + a b and acc + conj(a) b, each as four fused multiply-adds
template <typename C> __device__ __forceinline__ C cmac(C acc, C a, C b) {
    return mk(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
template <typename C> __device__ __forceinline__ C cmac_conj(C acc, C a, C b) {
    return mk(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}

// 2^x by the hardware's approximate base-2 exponential (PTX ex2.approx, results
// below the normal range flushed to zero): for the per-cell terms of the
// p-norm sums, each at most 1 and summed in FP32.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return mk(a.x * s, a.y * s); }
// multiply by +j
template <typename C> __device__ __forceinline__ C cmulj(C a) { return mk(-a.y, a.x); }

// ------------------------------------------------------- double-float sums --
// A value kept as hi + lo in two FP32 words (|lo| <= ulp(hi)/2).  Sums of
// FP32 partials in this form keep about 44 significant bits using FP32
// instructions only.  On this GPU the FP64 pipe is a latency trap on the
// per-evaluation critical path: a dependent FP64 add or FMA takes about ten
// times an FP32 one and an FP64 division or square root hundreds of cycles,
// and its throughput is a few operations per clock per SM.
struct __align__(8) DFloat {
    float hi, lo;
};

// Knuth's TwoSum of the high words (exact: s + e = a.hi + b.hi), then the
// low words folded in and the result renormalised.  The _rn intrinsics keep
// the compiler from contracting or reassociating the steps.
__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ DFloat df_warp_sum(DFloat a) {
    for (int o = 16; o > 0; o >>= 1) {
        const DFloat b = {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        a = df_add(a, b);
    }
    return a;
}
__device__ __forceinline__ double df_to_double(DFloat a) { return (double)a.hi + (double)a.lo; }

// The product of two FP32 values as an unevaluated pair p + e, exactly
// (Dekker's TwoProduct with a fused multiply-add: e = fma(a, b, -p) is the
// rounding error of p = a b, representable because an FP32 product has at
// most 48 significant bits).
__device__ __forceinline__ DFloat df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// Accumulate sum_n x(n) conj(h(n)) = (xr hr + xi hi) + j (xi hr - xr hi)
// with every product exact and the sums in double-float.
__device__ __forceinline__ void df_acc_xconjh(float2 xv, float2 hv, DFloat& sr, DFloat& si) {
    sr = df_add(sr, df_two_prod(xv.x, hv.x));
    sr = df_add(sr, df_two_prod(xv.y, hv.y));
    si = df_add(si, df_two_prod(xv.y, hv.x));
    si = df_add(si, df_two_prod(-xv.x, hv.y));
}

// chi_mm(0, 0) = sum_n x(n) conj(h(n)) (Eq. 38) by the NT threads of a CTA
// (all of them call it; it synchronises the CTA once): exact FP32 products,
// per-thread double-float partials, then a double-float tree (about 44
// significant bits in all); thread 0 stores the sum.
template <int NT>
__device__ __forceinline__ void diag_sum_f32(const float2* __restrict__ x, const float2* __restrict__ h, int N,
                                             double2* out) {
    __shared__ DFloat red[2][NT / 32];
    const int tid = threadIdx.x;
    DFloat sr = {0.f, 0.f}, si = {0.f, 0.f};
    for (int n = tid; n < N; n += NT) df_acc_xconjh(x[n], h[n], sr, si);
    const DFloat r = df_warp_sum(sr), i = df_warp_sum(si);
    if ((tid & 31) == 0) { red[0][tid >> 5] = r; red[1][tid >> 5] = i; }
    __syncthreads();
    if (tid == 0) {
        DFloat tr = red[0][0], ti = red[1][0];
        for (int w = 1; w < NT / 32; ++w) { tr = df_add(tr, red[0][w]); ti = df_add(ti, red[1][w]); }
        *out = make_double2(df_to_double(tr), df_to_double(ti));
    }
}

// e^{+j 2 pi s / 16} for s = 0..7 (cos, sin of multiples of pi/8).
__device__ __forceinline__ constexpr double w16c(int s) {
    return s == 0 ? 1.0 : s == 1 ? 0.92387953251128675613 : s == 2 ? 0.70710678118654752440
         : s == 3 ? 0.38268343236508977173 : s == 4 ? 0.0 : s == 5 ? -0.38268343236508977173
         : s == 6 ? -0.70710678118654752440 : -0.92387953251128675613;
}
__device__ __forceinline__ constexpr double w16s(int s) {
    return s == 0 ? 0.0 : s == 1 ? 0.38268343236508977173 : s == 2 ? 0.70710678118654752440
         : s == 3 ? 0.92387953251128675613 : s == 4 ? 1.0 : s == 5 ? 0.92387953251128675613
         : s == 6 ? 0.70710678118654752440 : 0.38268343236508977173;
}

// e^{+j 2 pi s / 32} for s = 1, 3, 5, ..., 15 (odd multiples of pi/16).
__device__ __forceinline__ constexpr double w32c(int s) {
    return s == 1 ? 0.980785280403230449126 : s == 3 ? 0.831469612302545237079 : s == 5 ? 0.555570233019602224743
         : s == 7 ? 0.195090322016128267848 : s == 9 ? -0.195090322016128267848
         : s == 11 ? -0.555570233019602224743 : s == 13 ? -0.831469612302545237079 : -0.980785280403230449126;
}
__device__ __forceinline__ constexpr double w32s(int s) {
    return s == 1 ? 0.195090322016128267848 : s == 3 ? 0.555570233019602224743 : s == 5 ? 0.831469612302545237079
         : s == 7 ? 0.980785280403230449126 : s == 9 ? 0.980785280403230449126
         : s == 11 ? 0.831469612302545237079 : s == 13 ? 0.555570233019602224743 : 0.195090322016128267848;
}

__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// Packed FP32 pairs (two lanes per instruction, one issue slot; the same
// IEEE round-to-nearest results as the scalar operations): e + o, and e - o
// as e + (-1) o (exact).  Used for the butterflies' plain additions: packed
// fused multiply-adds with constant pairs measured slower than the scalar
// tangent-form butterflies below (2048-bin rows: 217 us with packed additions
// only, 248 us with the twiddled butterflies packed as well).
__device__ __forceinline__ float2 padd(float2 e, float2 o) { return __fadd2_rn(e, o); }
__device__ __forceinline__ float2 psub(float2 e, float2 o) { return __ffma2_rn(o, make_float2(-1.f, -1.f), e); }

// One radix-2 butterfly with a compile-time twiddle, tp = e + w o and
// tm = e - w o for w = e^{+j 2 pi S / R}, with the multiplications folded into
// fused multiply-adds: six operations where a complex multiply and two
// complex additions take eight.  A general w = (c, s) is applied as
// c (o.x - t o.y, o.y + t o.x) with t = s/c when |c| >= |s|, else as
// s (u o.x - o.y, o.x + u o.y) with u = c/s (the tangent form of the
// rotation), so neither ratio exceeds 1.
template <int R, int S, typename C>
__device__ __forceinline__ void bfly_const(C e, C o, C& tp, C& tm) {
    using T = decltype(o.x);
    constexpr int s32 = S * (32 / R);
    if constexpr (sizeof(T) == 4 && s32 == 0) {
        tp = padd(e, o);                          // FP32 plain butterfly: packed pairs
        tm = psub(e, o);
    } else if constexpr (s32 == 0) {
        tp = cadd(e, o);
        tm = csub(e, o);
    } else if constexpr (s32 == 8) {            // w = j: w o = (-o.y, o.x)
        tp = mk(e.x - o.y, e.y + o.x);
        tm = mk(e.x + o.y, e.y - o.x);
    } else if constexpr (s32 == 4 || s32 == 12) {
        constexpr T r2 = (T)0.70710678118654752440;
        const T d = o.x - o.y, u = o.x + o.y;
        if constexpr (s32 == 4) {               // w o = r2 (o.x - o.y, o.x + o.y)
            tp = mk(fmadd(r2, d, e.x), fmadd(r2, u, e.y));
            tm = mk(fmadd(-r2, d, e.x), fmadd(-r2, u, e.y));
        } else {                                // w o = r2 (-(o.x + o.y), o.x - o.y)
            tp = mk(fmadd(-r2, u, e.x), fmadd(r2, d, e.y));
            tm = mk(fmadd(r2, u, e.x), fmadd(-r2, d, e.y));
        }
    } else {
        constexpr double cw = (s32 & 1) ? w32c(s32) : w16c(s32 / 2);
        constexpr double sw = (s32 & 1) ? w32s(s32) : w16s(s32 / 2);
        constexpr bool by_cos = (cw >= 0 ? cw : -cw) >= (sw >= 0 ? sw : -sw);
        T a, b;
        constexpr T f = (T)(by_cos ? cw : sw);
        if constexpr (by_cos) {
            constexpr T t = (T)(sw / cw);
            a = fmadd(-t, o.y, o.x);
            b = fmadd(t, o.x, o.y);
        } else {
            constexpr T u = (T)(cw / sw);
            a = fmadd(u, o.x, -o.y);
            b = fmadd(u, o.y, o.x);
        }
        tp = mk(fmadd(f, a, e.x), fmadd(f, b, e.y));
        tm = mk(fmadd(-f, a, e.x), fmadd(-f, b, e.y));
    }
}

// In-place R-point DFT with positive exponent, X[s] = sum_r v[r] e^{+j2 pi r s/R},
// on the elements v[0], v[ST], ..., v[(R-1) ST]; natural-order output.
// Radix-2 decimation in time, fully unrolled at compile time.
template <int R, int ST> struct Dft {
    template <typename C>
    static __device__ __forceinline__ void run(C* v) {
        Dft<R / 2, 2 * ST>::run(v);
        Dft<R / 2, 2 * ST>::run(v + ST);
        C t[R];
        combine<0>(v, t);
#pragma unroll
        for (int s = 0; s < R; ++s) v[ST * s] = t[s];
    }
    template <int S, typename C>
    static __device__ __forceinline__ void combine(const C* v, C* t) {
        if constexpr (S < R / 2) {
            bfly_const<R, S>(v[2 * ST * S], v[ST + 2 * ST * S], t[S], t[S + R / 2]);
            combine<S + 1>(v, t);
        }
    }
};
template <int ST> struct Dft<1, ST> {
    template <typename C> static __device__ __forceinline__ void run(C*) {}
};

// ----------------------------------------------------------- FFT plan ------
// L = E^a * r (E = 8 or 16 values per thread, r a smaller power of two), so
// T = L/E threads own one row.  Pass p has radix R(p) (E, then the
// remainder) and NS(p) = product of the previous radices.  Stockham
// auto-sort: after the last pass thread t holds bins b + r*NS_last for
// b = t + T*s, in natural order.
constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

template <int L, int E> struct Plan {
    static_assert(E == 8 || E == 16 || E == 32, "E must be 8, 16 or 32");
    static_assert(L >= 2 * E && L <= 4096 && (L & (L - 1)) == 0, "L must be a power of two in [2E, 4096]");
    static constexpr int T = L / E;
    static constexpr int lgE = ilog2c(E);
    static constexpr int nfull = ilog2c(L) / lgE;
    static constexpr int rem = 1 << (ilog2c(L) - nfull * lgE);
    static constexpr int passes = nfull + (rem > 1 ? 1 : 0);
    static constexpr int radix(int p) { return p < nfull ? E : rem; }
    static constexpr int ns(int p) { return p == 0 ? 1 : ns(p - 1) * radix(p - 1); }
    // offset of pass p's twiddle table [R-1][NS] for r = 1..R-1 (row r = 0 is all
    // ones and is not stored; pass 0 has no table)
    static constexpr int tw_off(int p) { return p <= 1 ? 0 : tw_off(p - 1) + (radix(p - 1) - 1) * ns(p - 1); }
    static constexpr int tw_len = tw_off(passes - 1) + (radix(passes - 1) - 1) * ns(passes - 1);
    static constexpr int padlen = L + L / E;       // row buffer with one pad slot per E
};

// Padded buffer index: one unused slot after every E entries, which makes
// the strided exchanges below free of shared-memory bank conflicts.
template <int E> __device__ __forceinline__ int padE(int i) { return i + (i >> ilog2c(E)); }

// Twiddle multiply + radix-R butterflies of pass (R, NS) on registers.
template <int L, int E, int R, int NS, typename C>
__device__ __forceinline__ void pass_compute(C (&v)[E], int t, const C* tw) {
    constexpr int T = L / E, NB = E / R;
#pragma unroll
    for (int s = 0; s < NB; ++s) {
        if constexpr (NS > 1) {
            const C* tk = tw + ((t + T * s) & (NS - 1));
#pragma unroll
            for (int r = 1; r < R; ++r) v[s * R + r] = cmul(v[s * R + r], tk[(r - 1) * NS]);
        }
        Dft<R, 1>::run(&v[s * R]);
    }
}

// Stockham write of a pass's outputs: value r of butterfly b goes to
// (b/NS) NS R + (b mod NS) + r NS.  Pass 0 (NS = 1) has R = E and every later
// pass has NS a multiple of E, so the padded address is a per-butterfly base
// plus a compile-time offset.
template <int L, int E, int R, int NS, typename C>
__device__ __forceinline__ void pass_store(const C (&v)[E], int t, C* buf) {
    constexpr int T = L / E, NB = E / R;
    static_assert(NS == 1 || NS % E == 0, "pass layout");
#pragma unroll
    for (int s = 0; s < NB; ++s) {
        const int b = t + T * s;
        C* p;
        if constexpr (NS == 1) {
            static_assert(R == E, "pass 0 has radix E");
            p = buf + b * (E + 1);
#pragma unroll
            for (int r = 0; r < R; ++r) p[r] = v[s * R + r];
        } else {
            const int base = (b / NS) * NS * R + (b & (NS - 1));
            p = buf + padE<E>(base);
#pragma unroll
            for (int r = 0; r < R; ++r) p[r * (NS / E) * (E + 1)] = v[s * R + r];
        }
    }
}

// Stockham read of a pass's inputs: value r of butterfly b is at b + r L/R.
template <int L, int E, int R, typename C>
__device__ __forceinline__ void pass_load(C (&v)[E], int t, const C* buf) {
    constexpr int T = L / E, NB = E / R, ST = L / R;
    if constexpr (ST % E == 0 && T % E == 0) {
        const C* p = buf + padE<E>(t);
#pragma unroll
        for (int s = 0; s < NB; ++s)
#pragma unroll
            for (int r = 0; r < R; ++r) v[s * R + r] = p[(T * s + r * ST) / E * (E + 1)];
    } else {
#pragma unroll
        for (int s = 0; s < NB; ++s)
#pragma unroll
            for (int r = 0; r < R; ++r) v[s * R + r] = buf[padE<E>(t + T * s + r * ST)];
    }
}

// Synchronise the T threads that own one row (a warp or a named barrier).
template <int T>
__device__ __forceinline__ void row_sync(int slot) {
    if constexpr (T <= 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(T) : "memory");
    }
}

// Passes 1..P-1 (pass 0 has been computed into v by the caller).
template <int L, int E, int P, typename C>
__device__ __forceinline__ void fft_rest(C (&v)[E], int t, int slot, C* buf, const C* tw) {
    using PL = Plan<L, E>;
    if constexpr (P < PL::passes) {
        constexpr int Rp = PL::radix(P - 1), NSp = PL::ns(P - 1);
        constexpr int R = PL::radix(P), NS = PL::ns(P);
        pass_store<L, E, Rp, NSp>(v, t, buf);
        row_sync<PL::T>(slot);
        pass_load<L, E, R>(v, t, buf);
        row_sync<PL::T>(slot);
        pass_compute<L, E, R, NS>(v, t, tw + PL::tw_off(P));
        fft_rest<L, E, P + 1>(v, t, slot, buf, tw);
    }
}

}  // namespace af

namespace af {
// Raise a kernel's dynamic shared-memory limit to the largest size requested
// so far on the current device (no-op afterwards, so it is safe to call while
// a stream is being captured once the first uncaptured launch has happened).
// The table is shared by every host thread and guarded by a lock.
inline cudaError_t set_smem_once(const void* func, int bytes) {
    struct Entry { const void* f; int dev; int bytes; };
    static Entry table[256];
    static int n = 0;
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < n; ++i)
        if (table[i].f == func && table[i].dev == dev && table[i].bytes >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < n; ++i)
        if (table[i].f == func && table[i].dev == dev) { table[i].bytes = bytes; return cudaSuccess; }
    if (n < 256) table[n++] = Entry{func, dev, bytes};
    return cudaSuccess;
}
}  // namespace af

namespace af {
// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may start before the kernel ahead of it in
// the stream has finished; pdl_wait() blocks until that kernel has completed
// and its memory is visible (a no-op when there is no such dependency), and
// pdl_trigger() lets the next kernel in the stream start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch `kern` with optional programmatic stream serialisation.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                             Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
}  // namespace af
