// af_noalloc.cu -- loss terms of one evaluation without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is
// being captured into a CUDA graph (an allocation would break the capture),
// hosts whose framework owns the device memory pool and forbids raw device
// allocations, and latency-critical loops that cannot afford the implicit
// synchronisation an allocation may cause.  af_loss_terms_noalloc serves
// them: it runs the same forward and finish kernels as af_loss_grad_xh, but
// every piece of scratch -- the FFT twiddle and phase tables, the per-CTA
// sidelobe partials and the per-waveform A_mm(0,0) -- lives in one
// file-scope __device__ array of fixed size, so nothing is allocated.
//
// Limits: the scratch is sized for L <= 4096 Doppler bins, N <= 4096 chips,
// M <= 16 waveforms and at most kMaxCtas forward CTAs (the launch geometry
// below keeps to that); larger problems are rejected with AF_ERR_INVALID_ARG.
// The array occupies kScratchBytes on every GPU that loads the library,
// until the process exits.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (a host-side name is not a device address); make
// that first call before any stream capture.  Every call shares the one
// array, which keeps the previous call's contents: calls that overlap on
// the GPU (different streams, or concurrent host threads) race.  Each call
// rewrites every scratch entry it reads before reading it, so nothing needs
// clearing between calls.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/sqngd.h"
#include "af_common.cuh"
#include "af_kernels.h"
#include "af_step.cuh"

namespace af {
namespace {

constexpr int kMaxL = 4096;
constexpr int kMaxN = 4096;
constexpr int kMaxM = 16;
constexpr int kMaxTw = 2 * kMaxL;          // any radix plan stores < 2L twiddles
constexpr int kMaxCtas = 8192;
constexpr int kMaxPasses = 8;

// byte offsets inside the scratch array (each region 256-byte aligned)
constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffTw = 0;
constexpr size_t kOffWL = align256(kOffTw + sizeof(float2) * kMaxTw);
constexpr size_t kOffPre = align256(kOffWL + sizeof(float2) * kMaxL);
constexpr size_t kOffKey = align256(kOffPre + sizeof(float2) * kMaxN);
constexpr size_t kOffIdx = align256(kOffKey + sizeof(float) * kMaxCtas);
constexpr size_t kOffChi = align256(kOffIdx + sizeof(long long) * kMaxCtas);
constexpr size_t kOffDiag = align256(kOffChi + sizeof(float2) * kMaxCtas);
constexpr size_t kScratchBytes = align256(kOffDiag + sizeof(double2) * kMaxM);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct PassTable {
    int n;
    int R[kMaxPasses];
    int NS[kMaxPasses];
};

// Twiddles (r = 1..R-1 rows of each pass p >= 1), e^{j 2 pi i / L} and the
// grid offset e^{j 2 pi nu0 n}, in FP64 then rounded, as the context builds them.
__global__ void fill_tables_kernel(float2* tw, float2* wL, float2* pre, PassTable pt, int L, int N, double nu0) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    int off = 0;
    for (int p = 1; p < pt.n; ++p) {
        const int R = pt.R[p], NS = pt.NS[p];
        for (int i = gid; i < (R - 1) * NS; i += stride) {
            const int r = i / NS + 1, k = i % NS;
            double sn, cs;
            sincospi(2.0 * (double)r * k / ((double)NS * R), &sn, &cs);
            tw[off + i] = make_float2((float)cs, (float)sn);
        }
        off += (R - 1) * NS;
    }
    for (int i = gid; i < L; i += stride) {
        double sn, cs;
        sincospi(2.0 * (double)i / L, &sn, &cs);
        wL[i] = make_float2((float)cs, (float)sn);
    }
    for (int n = gid; n < N; n += stride) {
        double t = nu0 * (double)n;
        t -= floor(t);
        double sn, cs;
        sincospi(2.0 * t, &sn, &cs);
        pre[n] = make_float2((float)cs, (float)sn);
    }
}

unsigned char* g_scratch_ptr[64];   // device address of the array, per device (set once, under g_setup)
std::mutex g_setup;

// The calling thread's failure message (af_last_error(NULL)), then the status.
af_status fail(af_status st, const char* fmt, const char* what) {
    char b[320];
    snprintf(b, sizeof b, fmt, what);
    set_thread_error(b);
    return st;
}

}  // namespace
}  // namespace af

using namespace af;

extern "C" af_status af_loss_terms_noalloc(int32_t M, int32_t N, int32_t L, double nu0, int32_t k_lo,
                                           int32_t k_hi, double eps, double snrl_db, const float* x_dev,
                                           const float* h_dev, double* terms_dev, void* stream) {
    auto bad = [](const char* m) { return fail(AF_ERR_INVALID_ARG, "af_loss_terms_noalloc: %s", m); };
    if (!x_dev || !h_dev || !terms_dev) return bad("x, h and terms must not be NULL");
    if (M < 1 || M > kMaxM) return bad("M must be in 1..16");
    if (N < 2 || N > kMaxN) return bad("N must be in 2..4096");
    if (L < 32 || L > kMaxL || (L & (L - 1)) != 0) return bad("L must be a power of two in 32..4096");
    if (k_lo < -(N - 1) || k_hi > N - 1 || k_lo > k_hi) return bad("delay window outside [-(N-1), N-1]");
    if (!(eps >= 0.0 && eps <= 1.0) || !(snrl_db >= 0.0) || !isfinite(nu0)) return bad("bad eps, snrl_db or nu0");
    const int E = fft_default_elems(L, false);
    // geometry: at most 32 delay chunks per pair
    const int D = k_hi - k_lo + 1;
    const int RS = fft_rows_per_cta(L, E);
    int rows = (D + 31) / 32;
    rows = ((rows + RS - 1) / RS) * RS;
    const int n_chunks = (D + rows - 1) / rows;
    const int nblk = M * M * n_chunks;
    if (nblk > kMaxCtas) return bad("too many forward CTAs for the scratch array");
    const int smem = fft_smem_bytes(L, N, false, E, 256, rows);
    if (smem <= 0 || smem > 227 * 1024) return bad("the forward pass does not fit in shared memory for this N, L");
    cudaStream_t s = (cudaStream_t)stream;

    // once per device: the array's device address
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(AF_ERR_CUDA, "af_loss_terms_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(AF_ERR_CUDA, "af_loss_terms_noalloc: %s", "device ordinal above 63");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup);
        if (g_scratch_ptr[dev] == nullptr) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || p == nullptr)
                return fail(AF_ERR_CUDA, "af_loss_terms_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch_ptr[dev] = (unsigned char*)p;
        }
        base = g_scratch_ptr[dev];
    }
    // the shared-memory limit of this (L, E) instantiation (a no-op once raised)
    e = fft_prepare_f32(L, N, E, 256, rows);
    if (e != cudaSuccess) return fail(AF_ERR_CUDA, "af_loss_terms_noalloc: kernel attribute: %s", cudaGetErrorString(e));
    float2* tw = (float2*)(base + kOffTw);
    float2* wL = (float2*)(base + kOffWL);
    float2* pre = (float2*)(base + kOffPre);
    float* pkey = (float*)(base + kOffKey);
    long long* pidx = (long long*)(base + kOffIdx);
    float2* pchi = (float2*)(base + kOffChi);
    double2* cdiag = (double2*)(base + kOffDiag);

    // radix plan of the FFT (radix-E passes, then the remainder)
    PassTable pt{};
    {
        int rem = L, ns = 1;
        while (rem >= E && rem % E == 0 && pt.n < kMaxPasses) { pt.R[pt.n] = E; pt.NS[pt.n] = ns; ++pt.n; ns *= E; rem /= E; }
        if (rem > 1) { pt.R[pt.n] = rem; pt.NS[pt.n] = ns; ++pt.n; }
    }
    fill_tables_kernel<<<32, 256, 0, s>>>(tw, wL, pre, pt, L, N, nu0);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        FwdArgs<float2, float> a{};
        a.M = M; a.N = N; a.L = L; a.D = D; a.k_lo = k_lo;
        a.n_chunks = n_chunks; a.rows_per_chunk = rows;
        a.x = (const float2*)x_dev; a.h = (const float2*)h_dev; a.pre = pre; a.tw = tw;
        a.weight_mode = WM_UNIFORM; a.mode = FWD_REDUCE; a.half_p = 0.f;
        a.pkey = pkey; a.pidx = pidx; a.pchi = pchi; a.cdiag = cdiag; a.fft_e = E;
        e = launch_fwd_fft_f32(a, s);
    }
    if (e == cudaSuccess) {
        FinArgs f{};
        f.M = M; f.N = N; f.L = L; f.D = D; f.k_lo = k_lo;
        f.nblk = nblk; f.ctas_per_pair = n_chunks;
        f.pkey = pkey; f.pidx = pidx; f.pchi = pchi; f.cdiag = cdiag;
        f.weight_mode = WM_UNIFORM; f.w0 = (float)(1.0 / N);
        f.eps = eps; f.ptar = pow(10.0, -snrl_db / 20.0); f.inv_N = 1.0 / N;
        f.snrl_coef = (1.0 - eps) * (2.0 / M) / N;
        f.grid_fft = 1; f.pre = pre; f.wL = wL;
        f.x = (const float2*)x_dev; f.h_in = (const float2*)h_dev;
        f.mode = FIN_GRAD_XH; f.terms = terms_dev;
        e = launch_fin(f, s);
    }
    if (e != cudaSuccess) return fail(AF_ERR_CUDA, "af_loss_terms_noalloc: launch: %s", cudaGetErrorString(e));
    set_thread_error("");
    return AF_OK;
}
