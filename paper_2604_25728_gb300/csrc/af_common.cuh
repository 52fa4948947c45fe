// af_common.cuh -- complex helpers, register DFTs and shared-memory Stockham
// passes used by the ambiguity-function kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return mk(a.x * s, a.y * s); }
// multiply by +j
template <typename C> __device__ __forceinline__ C cmulj(C a) { return mk(-a.y, a.x); }

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

// Multiply o by e^{+j 2 pi s / R} (s < R/2, R <= 16), folding the trivial cases.
template <int R, int S, typename C>
__device__ __forceinline__ C twiddle_const(C o) {
    using T = decltype(o.x);
    constexpr int s16 = S * (16 / R);
    if constexpr (s16 == 0) return o;
    else if constexpr (s16 == 4) return cmulj(o);
    else if constexpr (s16 == 2 || s16 == 6) {
        constexpr T r2 = (T)0.70710678118654752440;
        // e^{j pi/4} = r2 (1 + j); e^{j 3pi/4} = r2 (-1 + j)
        if constexpr (s16 == 2) return mk((o.x - o.y) * r2, (o.x + o.y) * r2);
        else return mk((-o.x - o.y) * r2, (o.x - o.y) * r2);
    } else {
        return cmul(o, mk((T)w16c(s16), (T)w16s(s16)));
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
            C e = v[2 * ST * S];
            C o = twiddle_const<R, S>(v[ST + 2 * ST * S]);
            t[S] = cadd(e, o);
            t[S + R / 2] = csub(e, o);
            combine<S + 1>(v, t);
        }
    }
};
template <int ST> struct Dft<1, ST> {
    template <typename C> static __device__ __forceinline__ void run(C*) {}
};

// ----------------------------------------------------------- FFT plan ------
// L = 16^a * r with r in {1, 2, 4, 8}; E = 16 values per thread, T = L/16
// threads per row; pass p has radix R(p) and NS(p) = product of the previous
// radices.  Stockham auto-sort: the output of the last pass is in natural
// order, thread t holding bins b + r*NS_last for b = t + T*s.
template <int L> struct Plan {
    static_assert(L >= 32 && L <= 4096 && (L & (L - 1)) == 0, "L must be a power of two in [32, 4096]");
    static constexpr int E = 16;
    static constexpr int T = L / 16;
    static constexpr int n16 = (L >= 4096) ? 3 : (L >= 256) ? 2 : 1;
    static constexpr int rem = L / (n16 == 3 ? 4096 : n16 == 2 ? 256 : 16);  // 1, 2, 4 or 8
    static constexpr int passes = n16 + (rem > 1 ? 1 : 0);
    static constexpr int radix(int p) { return p < n16 ? 16 : rem; }
    static constexpr int ns(int p) { return p == 0 ? 1 : ns(p - 1) * radix(p - 1); }
    // offset of pass p's twiddle table [R][NS] (pass 0 has none)
    static constexpr int tw_off(int p) { return p <= 1 ? 0 : tw_off(p - 1) + radix(p - 1) * ns(p - 1); }
    static constexpr int tw_len = tw_off(passes - 1) + radix(passes - 1) * ns(passes - 1);
    static constexpr int padlen = L + L / 16;      // row buffer length with one pad per 16
};

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// Twiddle multiply + radix-R butterflies of pass (R, NS) on registers.
template <int L, int R, int NS, typename C>
__device__ __forceinline__ void pass_compute(C (&v)[16], int t, const C* tw) {
    constexpr int T = L / 16, NB = 16 / R;
#pragma unroll
    for (int s = 0; s < NB; ++s) {
        if constexpr (NS > 1) {
            const int k = (t + T * s) & (NS - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) v[s * R + r] = cmul(v[s * R + r], tw[r * NS + k]);
        }
        Dft<R, 1>::run(&v[s * R]);
    }
}

template <int L, int R, int NS, typename C>
__device__ __forceinline__ void pass_store(const C (&v)[16], int t, C* buf) {
    constexpr int T = L / 16, NB = 16 / R;
#pragma unroll
    for (int s = 0; s < NB; ++s) {
        const int b = t + T * s;
        const int base = (b / NS) * NS * R + (b & (NS - 1));
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad16(base + r * NS)] = v[s * R + r];
    }
}

template <int L, int R, typename C>
__device__ __forceinline__ void pass_load(C (&v)[16], int t, const C* buf) {
    constexpr int T = L / 16, NB = 16 / R;
#pragma unroll
    for (int s = 0; s < NB; ++s) {
        const int b = t + T * s;
#pragma unroll
        for (int r = 0; r < R; ++r) v[s * R + r] = buf[pad16(b + r * (L / R))];
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
template <int L, int P, typename C>
__device__ __forceinline__ void fft_rest(C (&v)[16], int t, int slot, C* buf, const C* tw) {
    using PL = Plan<L>;
    if constexpr (P < PL::passes) {
        constexpr int Rp = PL::radix(P - 1), NSp = PL::ns(P - 1);
        constexpr int R = PL::radix(P), NS = PL::ns(P);
        pass_store<L, Rp, NSp>(v, t, buf);
        row_sync<PL::T>(slot);
        pass_load<L, R>(v, t, buf);
        row_sync<PL::T>(slot);
        pass_compute<L, R, NS>(v, t, tw + PL::tw_off(P));
        fft_rest<L, P + 1>(v, t, slot, buf, tw);
    }
}

// Bin index held in v[s*R + r] after the last pass.
template <int L>
__device__ __forceinline__ int out_bin(int t, int s, int r) {
    using PL = Plan<L>;
    constexpr int R = PL::radix(PL::passes - 1), NS = PL::ns(PL::passes - 1);
    return t + PL::T * s + r * NS;
    (void)R;
}

}  // namespace af

namespace af {
// Raise a kernel's dynamic shared-memory limit to the largest size requested
// so far on the current device (no-op afterwards, so it is safe to call while
// a stream is being captured once the first uncaptured launch has happened).
inline cudaError_t set_smem_once(const void* func, int bytes) {
    struct Entry { const void* f; int dev; int bytes; };
    static Entry table[256];
    static int n = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
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
