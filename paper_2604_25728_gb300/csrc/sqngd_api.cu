// sqngd_api.cu -- the C ABI of include/sqngd.h: context, tables, workspace,
// entry points and the CUDA-graph replay of Algorithm 1's outer iteration.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/resnet.h"
#include "../../include/sqngd.h"
#include "af_kernels.h"
#include "af_step.cuh"

using namespace af;

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// e^{j 2 pi t}, t in cycles, integer part removed first (FP64 on the host).
inline void phasor(double t, double* re, double* im) {
    const double f = t - floor(t);
    *re = cos(kTwoPi * f);
    *im = sin(kTwoPi * f);
}

struct FftPassInfo { int R, NS; };

// Host mirror of the device FFT plan (radix-E passes, then the remainder).
std::vector<FftPassInfo> fft_plan(int L, int E) {
    std::vector<FftPassInfo> p;
    int rem = L, ns = 1;
    while (rem >= E && rem % E == 0) { p.push_back({E, ns}); ns *= E; rem /= E; }
    if (rem > 1) p.push_back({rem, ns});
    return p;
}

template <typename T> struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct af_ctx {
    af_config cfg{};
    std::vector<double> nu;
    std::vector<float> wmap_host;
    int D = 0, P = 0, K = 0, path = 0;
    bool grid_fft = false;
    double nu0 = 0.0;
    float w0 = 0.f;
    cudaStream_t stream = nullptr;     // caller's stream
    cudaStream_t cap = nullptr;        // own stream for graph capture/replay
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int device = 0;
    std::string err;

    // tables
    float2* pre = nullptr;     // [N] e^{j 2 pi nu0 n}
    float2* tw = nullptr;      // FFT twiddles
    float2* wL = nullptr;      // [L] e^{j 2 pi i / L}
    float2* E = nullptr;       // [N][L] e^{j 2 pi nu_j n} (DFT path)
    uint16_t* bimg = nullptr;  // BF16 hi/lo images of B_m = x_m E, rebuilt per evaluation (tensor-core path)
    int gemm_n_ct = 0, gemm_n_kc = 0;
    int gemm_lb = 0;                      // bins per column tile
    int gemm_spc = 32, gemm_sb = 2, gemm_sa = 2;   // samples per stage, B stages, A stages
    int gemm_tiles = 1;                   // pairs per CTA sharing each B stage
    unsigned long long gemm_timeout_ns = 2000000000ull;   // limit of every pipeline wait
    int gemm_test_stall = 0;              // failure-detection test hook (SQNGD_GEMM_TEST_STALL)
    int gemm_split_ctas = 0;              // split schedule: CTAs sharing the chunk work (0: one CTA per tile)
    long long gemm_split_work = 0;        // chunks of all tiles
    int gemm_max_pieces = 0, gemm_ntiles = 0;
    float* gemm_part = nullptr;           // [tiles][max pieces][2 LB][128] partial accumulators of shared tiles
    int* gemm_tile_cnt = nullptr;         // [tiles] arrivals at each shared tile
    double2* pre64 = nullptr;
    double2* tw64 = nullptr;
    double2* E64 = nullptr;
    float* wmap = nullptr;     // [D][L]
    float* rho = nullptr;      // [K]
    float2* level = nullptr;   // [B]
    double2* level64 = nullptr;

    // workspace
    int n_chunks = 0, rows_per_chunk = 0, nblk = 0, ctas_per_pair = 0;
    bool acc_fft = false;
    bool rho_uniform = true;   // thresholds are the default (i + 1/2)/K
    bool pdl = true;           // programmatic dependent launch between forward and finish kernels
    int fft_e = 0, acc_e = 0;  // FFT values per thread: FP32 path, FP64 acceptance
    int fft_nt = 256;          // threads per forward CTA (FP32 FFT path)
    int acc_n_chunks = 0, acc_rows_per_chunk = 0, acc_nblk = 0, acc_ctas_per_pair = 0;
    float* pkey = nullptr;
    long long* pidx = nullptr;
    float* pvmax = nullptr;
    float* psum = nullptr;
    float2* pchi = nullptr;    // [nblk] chi at each forward CTA's best cell
    float2* adj_part = nullptr;    // [adj grid][2][N] dense-adjoint partial rows (p-norm loss)
    int* adj_cls = nullptr;        // the winning class of the last dense adjoint
    int adj_nt = 256;              // threads per dense-adjoint CTA
    int adj_e = 0;                 // values per thread of the dense adjoint's transforms
    float2* tw_adj = nullptr;      // its twiddles (when they differ from the forward's)
    AdjGeom adj_geom{};            // dense-adjoint grid (the winning class only)
    float2* dense = nullptr;       // [2][M][N] summed dense sidelobe gradient
    double* pkey64 = nullptr;
    long long* pidx64 = nullptr;
    double2* cdiag = nullptr;
    float2* xs = nullptr;      // soft waveform
    rn_net* rn = nullptr;      // attached transmit generator (Eq. 17), or null
    const float* rn_y0 = nullptr;
    float* du = nullptr;       // [M][N] dL/du of a transmit evaluation (generator)
    long long* rho_acc = nullptr;  // [K] fixed-point dL/drho accumulator (kept zeroed)
    float* m_rho = nullptr;    // [K] Adam moments of the trained thresholds
    float* v_rho = nullptr;
    float* gy = nullptr;       // [M][N] dL/dy and z of the last transmit evaluation (trained thresholds)
    float* zb = nullptr;
    float2* xs2 = nullptr;     // second soft buffer (matched mode: x_{j+1} is written while x_j is gathered)
    float* dydz = nullptr;
    float2* xh = nullptr;      // hard waveform
    double2* x64 = nullptr;
    double2* h64 = nullptr;
    double* acc_out = nullptr;
    double* terms_scratch = nullptr;
    int* errflag = nullptr;
    long long* ctr = nullptr;  // [4]
    double* best2 = nullptr;   // [8]
    double* log = nullptr;
    size_t log_cap_outer = 0;

    // sqngd_step graph cache
    cudaGraphExec_t gexec = nullptr;
    af_state gkey{};
    size_t g_log_cap = 0;
};

// messages of failures that have no context to hold them (af_init,
// af_loss_terms_noalloc), one per thread; af_last_error(NULL) returns it
static thread_local std::string g_init_error;

void af::set_thread_error(const char* msg) { g_init_error = msg ? msg : ""; }

#define FAIL(ctx, code, ...)                                        \
    do {                                                            \
        char _b[512];                                               \
        snprintf(_b, sizeof _b, __VA_ARGS__);                       \
        (ctx)->err = _b;                                            \
        return code;                                                \
    } while (0)

#define CK(ctx, call)                                                                      \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) FAIL(ctx, AF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
    } while (0)

template <typename T>
static af_status dalloc(af_ctx* c, T** p, size_t n) {
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        FAIL(c, e == cudaErrorMemoryAllocation ? AF_ERR_OOM : AF_ERR_CUDA, "cudaMalloc(%zu bytes): %s",
             n * sizeof(T), cudaGetErrorString(e));
    }
    return AF_OK;
}

template <typename T>
static af_status upload(af_ctx* c, T** p, const std::vector<T>& v) {
    af_status s = dalloc(c, p, v.size());
    if (s != AF_OK) return s;
    CK(c, cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return AF_OK;
}

static QuantArgs quant_args(const af_ctx* c) {
    QuantArgs q{};
    q.rho = c->rho;
    q.K = c->K;
    q.B = c->cfg.B;
    q.a = (float)(1.0 / (2.0 * c->cfg.B));
    q.c = (float)c->cfg.c;
    q.win = (float)(9.5 / c->cfg.c);     // tanh(9.5) rounds to 1 in FP32
    q.level = c->level;
    q.uniform = c->rho_uniform ? 1 : 0;
    return q;
}

static void free_all(af_ctx* c) {
    void* ptrs[] = {c->pre, c->tw, c->wL, c->E, c->pre64, c->tw64, c->E64, c->wmap, c->rho, c->level,
                    c->level64, c->pkey, c->pidx, c->pvmax, c->psum, c->pkey64, c->pidx64, c->cdiag,
                    c->xs, c->xs2, c->m_rho, c->v_rho, c->rho_acc, c->du, c->gy, c->zb, c->dydz, c->xh, c->x64, c->h64, c->acc_out, c->terms_scratch, c->errflag,
                    c->ctr, c->best2, c->log, c->pchi, c->adj_part, c->adj_cls, c->dense, c->tw_adj,
                    c->bimg, c->gemm_part, c->gemm_tile_cnt};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
}

// Rows per CTA for the FFT forward pass: every (pair, delay) row costs the
// same, a CTA takes RS rows per iteration, and `slots` CTAs are resident at
// once.  Choose the iteration count per CTA that minimises
// waves x (iterations + 1/2), the half iteration standing for the CTA's
// prologue (loading x, h and the twiddles).
// slots_of(it): resident CTAs on the whole GPU when a CTA's chunk holds it x RS
// rows (its shared memory grows with the chunk's h window).
template <typename SlotsOf>
static int pick_row_iters(int P, int D, int RS, SlotsOf slots_of) {
    int best_it = 1;
    double best_cost = 1e300;
    const int max_it = (D + RS - 1) / RS;
    for (int it = 1; it <= max_it; ++it) {
        int slots = slots_of(it);
        if (slots < 1) slots = 1;
        const long long rows = (long long)it * RS;
        const long long ctas = (long long)P * ((D + rows - 1) / rows);
        const long long waves = (ctas + slots - 1) / slots;
        const double cost = (double)waves * (it + 0.5);
        if (cost < best_cost) { best_cost = cost; best_it = it; }
    }
    return best_it;
}

static af_status validate(const af_config* g, std::string* why) {
    char b[256];
    auto bad = [&](const char* m) { *why = m; return AF_ERR_INVALID_ARG; };
    if (!g) return bad("cfg is NULL");
    if (g->M < 1 || g->M > 16) return bad("M must be in 1..16");
    if (g->N < 2 || g->N > 4096) return bad("N must be in 2..4096");
    if (g->B < 2 || g->B > 1024) return bad("B must be in 2..1024");
    if (g->L < 1 || g->L > 4096) return bad("L must be in 1..4096");
    if (!g->nu) return bad("nu is NULL");
    if (g->k_lo < -(g->N - 1) || g->k_hi > g->N - 1 || g->k_lo > g->k_hi) {
        snprintf(b, sizeof b, "delay window [%d, %d] outside [-(N-1), N-1] or empty", g->k_lo, g->k_hi);
        *why = b;
        return AF_ERR_INVALID_ARG;
    }
    if (!(g->eps >= 0.0 && g->eps <= 1.0)) return bad("eps must be in [0, 1]");
    if (!(g->snrl_db >= 0.0) || !isfinite(g->snrl_db)) return bad("snrl_db must be finite and >= 0");
    if (g->r_n < 1 || (long long)g->B * g->r_n > (1 << 20)) return bad("r_n must be >= 1 with B*r_n <= 2^20");
    if (!(g->c > 0.0) || !isfinite(g->c)) return bad("c must be finite and > 0");
    if (!(g->pnorm >= 0.0) || (g->pnorm > 0.0 && g->pnorm < 1.0)) return bad("pnorm must be 0 or >= 1");
    if (g->path < AF_PATH_AUTO || g->path > AF_PATH_SPLIT_BF16) return bad("unknown path");
    if (g->n_h < 0 || g->n_x < 0 || g->n_h + g->n_x < 1 || g->n_h + g->n_x > 256)
        return bad("n_h, n_x must be >= 0 with 1 <= n_h + n_x <= 256");
    if (g->matched != 0 && g->matched != 1) return bad("matched must be 0 or 1");
    if (g->matched && g->n_h != 0) return bad("matched (SQNAF) has no filter step: n_h must be 0");
    if (g->train_rho != 0 && g->train_rho != 1) return bad("train_rho must be 0 or 1");
    if (g->train_rho && (long long)g->B * g->r_n > 8192) return bad("train_rho needs K = B r_n <= 8192");
    if (g->train_rho && !(g->lr_rho >= 0.0 && isfinite(g->lr_rho))) return bad("lr_rho must be finite and >= 0");
    for (int j = 0; j < g->L; ++j)
        if (!isfinite(g->nu[j])) return bad("nu has a non-finite value");
    if (g->weights) {
        const long long n = (long long)(g->k_hi - g->k_lo + 1) * g->L;
        for (long long i = 0; i < n; ++i)
            if (!(g->weights[i] >= 0.f) || !isfinite(g->weights[i])) return bad("weights must be finite and >= 0");
    }
    return AF_OK;
}

extern "C" af_status af_init(const af_config* cfg, void* stream, af_ctx** out) {
    if (!out) { g_init_error = "out is NULL"; return AF_ERR_INVALID_ARG; }
    *out = nullptr;
    std::string why;
    if (validate(cfg, &why) != AF_OK) { g_init_error = why; return AF_ERR_INVALID_ARG; }

    af_ctx* c = new af_ctx();
    c->cfg = *cfg;
    c->cfg.nu = nullptr;
    c->cfg.weights = nullptr;
    if (c->cfg.beta1 == 0.0) c->cfg.beta1 = 0.9;
    if (c->cfg.beta2 == 0.0) c->cfg.beta2 = 0.999;
    if (c->cfg.adam_eps == 0.0) c->cfg.adam_eps = 1e-8;
    const int M = cfg->M, N = cfg->N, L = cfg->L;
    c->nu.assign(cfg->nu, cfg->nu + L);
    c->D = cfg->k_hi - cfg->k_lo + 1;
    c->P = M * M;
    c->K = cfg->B * cfg->r_n;
    c->w0 = (float)(1.0 / N);
    c->stream = (cudaStream_t)stream;
    if (const char* e = getenv("SQNGD_NO_PDL")) c->pdl = (atoi(e) == 0);
    auto fail = [&](af_status s) {
        g_init_error = c->err;
        free_all(c);
        delete c;
        return s;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) { c->err = "no CUDA device"; return fail(AF_ERR_CUDA); }

    // ---- grid: uniform with spacing 1/L (FFT-able) or arbitrary ----
    c->nu0 = c->nu[0];
    bool uniform = (L >= 32 && L <= 4096 && (L & (L - 1)) == 0);
    for (int j = 0; uniform && j < L; ++j)
        if (fabs(c->nu[j] - (c->nu0 + (double)j / L)) > 1e-12) uniform = false;
    c->fft_e = uniform ? fft_default_elems(L, false) : 0;
    // the dense adjoint of the p-norm loss is built for 8 and 16 values per
    // thread (it holds two transforms' operands and a gradient row in registers)
    c->adj_e = (c->fft_e == 32) ? 16 : c->fft_e;
    c->fft_nt = uniform ? fft_default_threads(L, c->fft_e, false) : 256;
    if (uniform && c->fft_nt != 256) {
        const int wide = fft_smem_bytes(L, N, false, c->fft_e, c->fft_nt);
        if (wide <= 0 || wide > 227 * 1024) c->fft_nt = 256;   // the wide CTA does not fit: 256 threads
    }
    const int fft_smem = uniform ? fft_smem_bytes(L, N, false, c->fft_e, c->fft_nt) : -1;
    uniform = uniform && fft_smem > 0 && fft_smem <= 227 * 1024;
    if (cfg->path == AF_PATH_FFT && !uniform) {
        c->err = "AF_PATH_FFT needs nu_j = nu_0 + j/L with L a power of two in 32..4096";
        return fail(AF_ERR_UNIMPLEMENTED);
    }
    c->path = (cfg->path == AF_PATH_AUTO) ? (uniform ? AF_PATH_FFT : AF_PATH_DFT) : cfg->path;
    if (c->path == AF_PATH_SPLIT_BF16) {
        if (const char* e = getenv("SQNGD_GEMM_CFG")) {   // "<samples per stage>x<B stages>x<A stages>"
            int a = 0, b = 0, d = 0;
            if (sscanf(e, "%dx%dx%d", &a, &b, &d) != 3) {
                c->err = "SQNGD_GEMM_CFG must read <samples per stage>x<B stages>x<A stages>";
                return fail(AF_ERR_INVALID_ARG);
            }
            c->gemm_spc = a; c->gemm_sb = b; c->gemm_sa = d;
        }
        const int P = M * M;
        c->gemm_tiles = 1;
        if (const char* e = getenv("SQNGD_GEMM_TILES")) {
            const int v = atoi(e);
            if ((v == 1 || v == 2) && P % v == 0) c->gemm_tiles = v;
        }
        // failure-detection test: every forward's MMA issuer waits on a barrier
        // that nothing completes, with a 50 ms limit
        if (const char* e = getenv("SQNGD_GEMM_TEST_STALL"))
            if (atoi(e) != 0) { c->gemm_test_stall = 1; c->gemm_timeout_ns = 50000000ull; }
        // Column tiles: the widest that covers L, narrowed (down to 16 bins)
        // while there are fewer tiles than a quarter of the SMs -- every column
        // tile is an independent part of the output, so narrower tiles add
        // CTAs without any merge (measured on M=4, N=1024, 128 bins, 101
        // delays: 128 bins per tile 36.5 us, 64 or 32 bins 29.4 us, 16 bins
        // 31.5 us per forward pass).
        {
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1)
                sms = 1;
            const int dtiles = (c->D + kGemmRows - 1) / kGemmRows;
            int lb = gemm_bins_per_tile(L);
            auto tiles_of = [&](int b) { return P / c->gemm_tiles * dtiles * ((L + b - 1) / b); };
            while (lb > 16 && 4 * tiles_of(lb) < sms) lb /= 2;
            if (const char* e = getenv("SQNGD_GEMM_LB")) {
                const int v = atoi(e);
                if ((v == 16 || v == 32 || v == 64 || v == 128) && v <= gemm_bins_per_tile(L)) lb = v;
            }
            c->gemm_lb = lb;
        }
        if (!gemm_shape_supported(c->gemm_lb, N, c->gemm_spc, c->gemm_sb, c->gemm_sa, c->gemm_tiles)) {
            c->err = "AF_PATH_SPLIT_BF16: pipeline shape does not fit this N and L";
            return fail(AF_ERR_UNIMPLEMENTED);
        }
        // Split schedule: with fewer tiles than SMs, the CTAs that fit at once
        // share the chunk work equally and tiles are split between them, so
        // no SM idles (measured on M=4, N=1024, 128 bins, 101 delays, 64 tiles
        // of 32 bins: 30.2 -> 27.2 us per forward pass).  With more tiles than
        // SMs it measured slower (256 tiles on 152 SMs: 38.5 -> 44.0 us): each
        // CTA then holds about two pieces, and a piece's window fill, partial
        // store and merge cost more than the balance gains.
        // SQNGD_GEMM_SPLIT=0 turns it off; SQNGD_GEMM_SPLIT_CTAS=n forces n
        // CTAs (tests of the schedule).
        {
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1)
                sms = 1;
            const int n_blocks = (c->D + kGemmRows - 1) / kGemmRows;
            const int n_ct = (L + c->gemm_lb - 1) / c->gemm_lb;
            const int ntile = P * n_blocks * n_ct;
            const int fit = sms * gemm_ctas_per_sm(c->gemm_lb, N, c->gemm_spc, c->gemm_sb, c->gemm_sa, 1);
            int ctas = (ntile < sms) ? fit : 0;
            if (const char* e = getenv("SQNGD_GEMM_SPLIT"))
                if (atoi(e) == 0) ctas = 0;
            if (const char* e = getenv("SQNGD_GEMM_SPLIT_CTAS")) ctas = atoi(e) > 0 ? atoi(e) : ctas;
            // built for one pair per CTA in the default pipeline shape
            if (c->gemm_tiles != 1 || c->gemm_spc != 32 || c->gemm_sb != 2 || c->gemm_sa != 2) ctas = 0;
            if (ctas > 0) {
                const GemmSplitPlan plan =
                    gemm_split_plan(P, n_blocks, n_ct, c->cfg.k_lo, c->D, N, c->gemm_spc, ctas);
                if (plan.ok) {
                    c->gemm_split_ctas = ctas;
                    c->gemm_split_work = plan.work;
                    c->gemm_max_pieces = plan.max_pieces;
                    c->gemm_ntiles = ntile;
                }
            }
        }
    }
    c->grid_fft = uniform;
    if (cfg->pnorm > 0.0) {
        // the dense adjoint of the p-norm loss runs on the FFT grid; its grid
        // spans the winning class only, its CTA as wide as shared memory allows
        int sms_a = 0;
        if (cudaDeviceGetAttribute(&sms_a, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms_a < 1)
            sms_a = 1;
        int adj = -1;
        for (int nt : {adj_threads(L, c->adj_e), 256}) {
            if (c->path != AF_PATH_FFT) break;
            c->adj_nt = nt;
            adj_geometry(M, c->D, L, c->adj_e, nt, sms_a, &c->adj_geom);
            adj = adj_smem_bytes(L, N, c->adj_e, nt, c->adj_geom.rpc_max);
            if (adj > 0 && adj <= 227 * 1024) break;
        }
        if (adj <= 0 || adj > 227 * 1024) {
            c->err = "pnorm > 0 needs the FFT path (uniform grid) with the adjoint fitting in shared memory";
            return fail(AF_ERR_UNIMPLEMENTED);
        }
    }
    // FP64 acceptance pass: FFT when it fits in shared memory
    c->acc_e = c->grid_fft ? fft_default_elems(L, true) : 0;
    {
        const int smem64 = c->grid_fft ? fft_smem_bytes(L, N, true, c->acc_e) : -1;
        c->acc_fft = c->grid_fft && smem64 > 0 && smem64 <= 227 * 1024;
    }

    af_status s;
    // ---- tables, built in FP64 ----
    std::vector<float2> pre(N), wL(L), lev(c->cfg.B);
    std::vector<double2> pre64(N), lev64(c->cfg.B);
    for (int n = 0; n < N; ++n) {
        double re, im;
        phasor(c->nu0 * n, &re, &im);
        pre[n] = make_float2((float)re, (float)im);
        pre64[n] = make_double2(re, im);
    }
    for (int i = 0; i < L; ++i) {
        double re, im;
        phasor((double)i / L, &re, &im);
        wL[i] = make_float2((float)re, (float)im);
    }
    for (int b = 0; b < c->cfg.B; ++b) {
        double re, im;
        phasor((double)b / c->cfg.B, &re, &im);
        lev[b] = make_float2((float)re, (float)im);
        lev64[b] = make_double2(re, im);
    }
    if ((s = upload(c, &c->pre, pre)) || (s = upload(c, &c->pre64, pre64)) || (s = upload(c, &c->wL, wL)) ||
        (s = upload(c, &c->level, lev)) || (s = upload(c, &c->level64, lev64)))
        return fail(s);
    // Stockham twiddles: for every pass p >= 1 a table [R-1][NS] of
    // e^{+j 2 pi r k / (NS R)}, r = 1..R-1 (the r = 0 row is all ones)
    auto twiddles = [&](int E, std::vector<double2>& out) {
        const auto plan = fft_plan(L, E);
        for (size_t p = 1; p < plan.size(); ++p) {
            const int R = plan[p].R, NS = plan[p].NS;
            for (int r = 1; r < R; ++r)
                for (int k = 0; k < NS; ++k) {
                    double re, im;
                    phasor((double)r * k / ((double)NS * R), &re, &im);
                    out.push_back(make_double2(re, im));
                }
        }
    };
    if (c->grid_fft) {
        std::vector<double2> t32, t64;
        twiddles(c->fft_e, t32);
        twiddles(c->acc_e, t64);
        std::vector<float2> tw(t32.size());
        for (size_t i = 0; i < t32.size(); ++i) tw[i] = make_float2((float)t32[i].x, (float)t32[i].y);
        if ((s = upload(c, &c->tw, tw)) || (s = upload(c, &c->tw64, t64))) return fail(s);
        if (cfg->pnorm > 0.0 && c->adj_e != c->fft_e) {
            std::vector<double2> ta;
            twiddles(c->adj_e, ta);
            std::vector<float2> twa(ta.size());
            for (size_t i = 0; i < ta.size(); ++i) twa[i] = make_float2((float)ta[i].x, (float)ta[i].y);
            if ((s = upload(c, &c->tw_adj, twa))) return fail(s);
        }
    }
    {
        // phasor table of the arbitrary-grid path (also used for acceptance when
        // the FP64 FFT does not fit in shared memory)
        std::vector<float2> E((size_t)N * L);
        std::vector<double2> E64((size_t)N * L);
        for (int n = 0; n < N; ++n)
            for (int j = 0; j < L; ++j) {
                double re, im;
                phasor(c->nu[j] * n, &re, &im);
                E[(size_t)n * L + j] = make_float2((float)re, (float)im);
                E64[(size_t)n * L + j] = make_double2(re, im);
            }
        if ((s = upload(c, &c->E, E)) || (s = upload(c, &c->E64, E64))) return fail(s);
    }
    if (c->path == AF_PATH_SPLIT_BF16) {
        if ((s = dalloc(c, &c->bimg, gemm_bimg_bytes(M, N, L, c->gemm_lb, c->gemm_spc) / sizeof(uint16_t))))
            return fail(s);
        if (c->gemm_split_ctas > 0) {
            const size_t np = (size_t)c->gemm_ntiles * c->gemm_max_pieces * (2 * c->gemm_lb) * kGemmRows;
            if ((s = dalloc(c, &c->gemm_part, np)) || (s = dalloc(c, &c->gemm_tile_cnt, (size_t)c->gemm_ntiles)))
                return fail(s);
            if (cudaMemset(c->gemm_tile_cnt, 0, sizeof(int) * c->gemm_ntiles) != cudaSuccess) {
                c->err = "cudaMemset failed";
                return fail(AF_ERR_CUDA);
            }
        }
        const int LB = c->gemm_lb;
        c->gemm_n_ct = (L + LB - 1) / LB;
        c->gemm_n_kc = (N + c->gemm_spc - 1) / c->gemm_spc;
    }
    if (cfg->weights) {
        c->wmap_host.assign(cfg->weights, cfg->weights + (size_t)c->D * L);
        if ((s = upload(c, &c->wmap, c->wmap_host))) return fail(s);
    }
    {
        std::vector<float> rho(c->K);
        for (int i = 0; i < c->K; ++i) rho[i] = (float)(((double)i + 0.5) / (double)c->K);
        if ((s = upload(c, &c->rho, rho))) return fail(s);
    }

    // ---- launch geometry and workspace ----
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1) sms = 1;
    if (c->path == AF_PATH_FFT) {
        const int RS = fft_rows_per_cta(L, c->fft_e, c->fft_nt);
        int it = pick_row_iters(c->P, c->D, RS, [&](int i) {
            return sms * fft_occupancy(L, N, c->fft_e, false, c->fft_nt, i * RS);
        });
        if (const char* e = getenv("SQNGD_FFT_ROW_ITERS")) it = atoi(e) > 0 ? atoi(e) : it;
        c->rows_per_chunk = RS * it;
        c->n_chunks = (c->D + c->rows_per_chunk - 1) / c->rows_per_chunk;
        c->ctas_per_pair = c->n_chunks;
    } else if (c->path == AF_PATH_SPLIT_BF16) {
        c->rows_per_chunk = kGemmRows;
        c->n_chunks = (c->D + kGemmRows - 1) / kGemmRows;
        c->ctas_per_pair = c->n_chunks * c->gemm_n_ct;
    } else {
        c->rows_per_chunk = dft_rows_per_cta(L);
        c->n_chunks = (c->D + c->rows_per_chunk - 1) / c->rows_per_chunk;
        c->ctas_per_pair = c->n_chunks * dft_col_tiles(L);
    }
    c->nblk = c->P * c->ctas_per_pair;
    if (c->acc_fft) {
        const int RS = fft_rows_per_cta(L, c->acc_e);
        const int it = pick_row_iters(c->P, c->D, RS, [&](int i) {
            return sms * fft_occupancy(L, N, c->acc_e, true, 256, i * RS);
        });
        c->acc_rows_per_chunk = RS * it;
        c->acc_n_chunks = (c->D + c->acc_rows_per_chunk - 1) / c->acc_rows_per_chunk;
        c->acc_ctas_per_pair = c->acc_n_chunks;
    } else {
        c->acc_rows_per_chunk = dft_rows_per_cta(L);
        c->acc_n_chunks = (c->D + c->acc_rows_per_chunk - 1) / c->acc_rows_per_chunk;
        c->acc_ctas_per_pair = c->acc_n_chunks * dft_col_tiles(L);
    }
    c->acc_nblk = c->P * c->acc_ctas_per_pair;

    // kernels' shared-memory limits are raised here, for this geometry, outside any graph capture
    {
        cudaError_t e = (c->path == AF_PATH_FFT) ? fft_prepare_f32(L, N, c->fft_e, c->fft_nt, c->rows_per_chunk)
                        : (c->path == AF_PATH_SPLIT_BF16) ? gemm_prepare(c->gemm_lb, N, c->gemm_spc, c->gemm_sb, c->gemm_sa, c->gemm_tiles)
                        : dft_prepare_f32(N);
        if (e == cudaSuccess)
            e = c->acc_fft ? fft_prepare_f64(L, N, c->acc_e, 256, c->acc_rows_per_chunk) : dft_prepare_f64(N);
        if (e == cudaSuccess && cfg->pnorm > 0.0) e = adj_prepare(L, N, c->adj_e, c->adj_nt, c->adj_geom.rpc_max);
        if (e == cudaSuccess && c->K <= 8192) e = rho_prepare(c->K);
        if (e != cudaSuccess) { c->err = std::string("kernel attribute: ") + cudaGetErrorString(e); return fail(AF_ERR_CUDA); }
    }
    const size_t MN = (size_t)M * N;
    if ((s = dalloc(c, &c->pkey, c->nblk)) || (s = dalloc(c, &c->pidx, c->nblk)) ||
        (s = dalloc(c, &c->pvmax, c->nblk)) || (s = dalloc(c, &c->psum, c->nblk)) ||
        (s = dalloc(c, &c->pchi, c->nblk)) ||
        (s = dalloc(c, &c->pkey64, c->acc_nblk)) || (s = dalloc(c, &c->pidx64, c->acc_nblk)) ||
        (s = dalloc(c, &c->cdiag, M)) || (s = dalloc(c, &c->xs, MN)) || (s = dalloc(c, &c->dydz, MN)) ||
        (cfg->matched && (s = dalloc(c, &c->xs2, MN))) ||
        (s = dalloc(c, &c->gy, MN)) || (s = dalloc(c, &c->zb, MN)) || (s = dalloc(c, &c->du, MN)) ||
        (cfg->train_rho && ((s = dalloc(c, &c->m_rho, c->K)) || (s = dalloc(c, &c->v_rho, c->K)))) ||
        (c->K <= 8192 && (s = dalloc(c, &c->rho_acc, c->K))) ||
        (s = dalloc(c, &c->xh, MN)) || (s = dalloc(c, &c->x64, MN)) || (s = dalloc(c, &c->h64, MN)) ||
        (s = dalloc(c, &c->acc_out, 4 + M)) || (s = dalloc(c, &c->terms_scratch, AF_TERMS_FIXED + M)) ||
        (s = dalloc(c, &c->errflag, 1)) || (s = dalloc(c, &c->ctr, 4)) || (s = dalloc(c, &c->best2, 8)))
        return fail(s);
    if (cfg->pnorm > 0.0 &&
        ((s = dalloc(c, &c->adj_part, (size_t)c->adj_geom.grid * 2 * N)) || (s = dalloc(c, &c->dense, 2 * MN)) ||
         (s = dalloc(c, &c->adj_cls, 1))))
        return fail(s);
    if (c->rho_acc && cudaMemset(c->rho_acc, 0, sizeof(long long) * c->K) != cudaSuccess) {
        c->err = "cudaMemset failed";
        return fail(AF_ERR_CUDA);
    }
    if (cfg->train_rho) {
        // trained thresholds leave the uniform set: every quantizer reads the table
        c->rho_uniform = false;
        if (cudaMemset(c->m_rho, 0, sizeof(float) * c->K) != cudaSuccess ||
            cudaMemset(c->v_rho, 0, sizeof(float) * c->K) != cudaSuccess) {
            c->err = "cudaMemset failed";
            return fail(AF_ERR_CUDA);
        }
    }
    if (cudaMemset(c->errflag, 0, sizeof(int)) != cudaSuccess) {
        c->err = "cudaMemset failed";
        return fail(AF_ERR_CUDA);
    }
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        c->err = "stream/event creation failed";
        return fail(AF_ERR_CUDA);
    }
    *out = c;
    return AF_OK;
}

extern "C" af_status af_destroy(af_ctx* c) {
    if (!c) return AF_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    cudaStreamSynchronize(c->cap);
    free_all(c);
    delete c;
    return AF_OK;
}

extern "C" const char* af_last_error(const af_ctx* c) { return c ? c->err.c_str() : g_init_error.c_str(); }

extern "C" int32_t af_path_of(const af_ctx* c) { return c ? c->path : -1; }

extern "C" af_status af_sync(af_ctx* c) {
    if (!c) return AF_ERR_INVALID_ARG;
    CK(c, cudaStreamSynchronize(c->stream));
    int flag = 0;
    CK(c, cudaMemcpy(&flag, c->errflag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CK(c, cudaMemset(c->errflag, 0, sizeof(int)));
        if (flag & 2) FAIL(c, AF_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
        FAIL(c, AF_ERR_NONFINITE, "a loss or gradient was NaN or Inf");
    }
    return AF_OK;
}

extern "C" af_status af_set_thresholds(af_ctx* c, const float* rho_host) {
    if (!c || !rho_host) return AF_ERR_INVALID_ARG;
    for (int i = 0; i < c->K; ++i) {
        if (!(rho_host[i] >= 0.f && rho_host[i] <= 1.f)) FAIL(c, AF_ERR_INVALID_ARG, "rho[%d] outside [0, 1]", i);
        if (i > 0 && !(rho_host[i] > rho_host[i - 1])) FAIL(c, AF_ERR_INVALID_ARG, "rho not strictly increasing at %d", i);
    }
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemcpy(c->rho, rho_host, sizeof(float) * c->K, cudaMemcpyHostToDevice));
    c->rho_uniform = false;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return AF_OK;
}

// ---------------------------------------------------------------- forward --
static FwdArgs<float2, float> fwd_args(af_ctx* c, const float2* x, const float2* h) {
    FwdArgs<float2, float> a{};
    a.M = c->cfg.M; a.N = c->cfg.N; a.L = c->cfg.L; a.D = c->D; a.k_lo = c->cfg.k_lo;
    a.n_chunks = c->n_chunks; a.rows_per_chunk = c->rows_per_chunk;
    a.x = x; a.h = h; a.pre = c->pre;
    a.tw = (c->path == AF_PATH_FFT) ? c->tw : c->E;
    a.wmap = c->wmap;
    a.weight_mode = c->wmap ? WM_MAP : WM_UNIFORM;
    a.mode = FWD_REDUCE;
    a.half_p = (float)(c->cfg.pnorm * 0.5);
    a.pkey = c->pkey; a.pidx = c->pidx; a.pvmax = c->pvmax; a.psum = c->psum; a.pchi = c->pchi;
    a.cdiag = c->cdiag;
    a.fft_e = c->fft_e;
    a.fft_nt = c->fft_nt;
    a.pdl = c->pdl ? 1 : 0;
    return a;
}

static cudaError_t launch_fwd(af_ctx* c, const FwdArgs<float2, float>& a, cudaStream_t s) {
    if (c->path == AF_PATH_SPLIT_BF16) {
        // this evaluation's B_m images, then the contraction
        cudaError_t e = launch_gemm_bimg(a.x, c->E, c->cfg.M, c->cfg.N, c->cfg.L, c->gemm_lb, c->gemm_spc, c->bimg,
                                         c->gemm_tile_cnt, c->gemm_ntiles, a.pdl, s);
        if (e != cudaSuccess) return e;
        GemmArgs g{};
        g.f = a;
        g.bimg = c->bimg;
        g.err = c->errflag;
        g.lb = c->gemm_lb;
        g.n_ct = c->gemm_n_ct;
        g.n_kc = c->gemm_n_kc;
        g.spc = c->gemm_spc;
        g.sb = c->gemm_sb;
        g.sa = c->gemm_sa;
        g.tiles = c->gemm_tiles;
        g.timeout_ns = c->gemm_timeout_ns;
        g.test_stall = c->gemm_test_stall;
        g.split_ctas = c->gemm_split_ctas;
        g.split_work = c->gemm_split_work;
        g.max_pieces = c->gemm_max_pieces;
        g.part = c->gemm_part;
        g.tile_cnt = c->gemm_tile_cnt;
        return launch_fwd_gemm(g, s);
    }
    return (c->path == AF_PATH_FFT) ? launch_fwd_fft_f32(a, s) : launch_fwd_dft_f32(a, s);
}

// The forward pass of one evaluation, followed for the p-norm loss by the
// dense adjoint (whose summed gradient the finish kernel then adds) unless
// no gradient is wanted (`adjoint` false: the loss terms alone).
static cudaError_t launch_eval_forward(af_ctx* c, const float2* x, const float2* h, cudaStream_t s,
                                       long long* ctr_inc, bool adjoint = true) {
    FwdArgs<float2, float> a = fwd_args(c, x, h);
    a.ctr_inc = ctr_inc;
    cudaError_t e = launch_fwd(c, a, s);
    if (e != cudaSuccess || !(c->cfg.pnorm > 0.0) || !adjoint) return e;
    AdjArgs d{};
    d.M = c->cfg.M; d.N = c->cfg.N; d.L = c->cfg.L; d.D = c->D; d.k_lo = c->cfg.k_lo;
    d.grid = c->adj_geom.grid;
    d.cpp_cls[0] = c->adj_geom.cpp[0]; d.cpp_cls[1] = c->adj_geom.cpp[1];
    d.rows_cls[0] = c->adj_geom.rows[0]; d.rows_cls[1] = c->adj_geom.rows[1];
    d.rpc_max = c->adj_geom.rpc_max;
    d.nt = c->adj_nt;
    d.cls_buf = c->adj_cls;
    d.x = x; d.h = h; d.pre = c->pre; d.tw = c->tw_adj ? c->tw_adj : c->tw;
    d.wmap = c->wmap; d.weight_mode = c->wmap ? WM_MAP : WM_UNIFORM; d.w0 = c->w0;
    d.eps = c->cfg.eps; d.half_p = (float)(c->cfg.pnorm * 0.5);
    d.nblk_fwd = c->nblk; d.ctas_per_pair_fwd = c->ctas_per_pair;
    d.pvmax = c->pvmax; d.psum = c->psum;
    d.part = c->adj_part; d.dense = c->dense;
    d.fft_e = c->adj_e; d.pdl = c->pdl ? 1 : 0;
    return launch_adj(d, s);
}

// Evaluations per outer iteration: Step A and Step B, or (matched) one score
// of the hard design and Step B.
static int evals_per_outer(const af_ctx* c) {
    return c->cfg.matched ? 1 + c->cfg.n_x : c->cfg.n_h + c->cfg.n_x;
}

static FinArgs fin_args(af_ctx* c) {
    FinArgs f{};
    f.M = c->cfg.M; f.N = c->cfg.N; f.L = c->cfg.L; f.D = c->D; f.k_lo = c->cfg.k_lo;
    f.nblk = c->nblk; f.ctas_per_pair = c->ctas_per_pair;
    f.pkey = c->pkey; f.pidx = c->pidx; f.pvmax = c->pvmax; f.psum = c->psum; f.pchi = c->pchi;
    f.cdiag = c->cdiag;
    f.weight_mode = c->wmap ? WM_MAP : WM_UNIFORM;
    f.w0 = c->w0; f.wmap = c->wmap;
    f.eps = c->cfg.eps;
    f.inv_N = 1.0 / c->cfg.N;
    f.pdl = c->pdl ? 1 : 0;
    f.ptar = pow(10.0, -c->cfg.snrl_db / 20.0);
    f.snrl_coef = (1.0 - c->cfg.eps) * (2.0 / c->cfg.M) / c->cfg.N;
    f.half_p = (float)(c->cfg.pnorm * 0.5);
    f.grid_fft = c->grid_fft ? 1 : 0;
    f.pre = c->pre; f.wL = c->wL; f.E = c->E;
    f.err_flag = c->errflag;
    f.qa = quant_args(c);
    f.snrl_db = c->cfg.snrl_db;
    {
        const double p = pow(10.0, -(c->cfg.snrl_db + 0.05) / 20.0);
        f.p_accept2 = p * p;
    }
    f.n_h = c->cfg.n_h; f.n_x = c->cfg.n_x;
    f.evals_per_outer = evals_per_outer(c);
    f.matched = c->cfg.matched;
    if (c->cfg.pnorm > 0.0) { f.dense_g = c->dense; f.n_dense = 1; }
    f.lr = 0.f;
    f.b1 = (float)c->cfg.beta1; f.b2 = (float)c->cfg.beta2; f.adam_eps = (float)c->cfg.adam_eps;
    return f;
}

// Arguments of the threshold kernel for this context.
static RhoArgs rho_args(af_ctx* c, int mode) {
    RhoArgs r{};
    r.mode = mode;
    r.n = c->cfg.M * c->cfg.N;
    r.gy = c->gy; r.z = c->zb;
    r.q = quant_args(c);
    r.rho = c->rho;
    r.acc = c->rho_acc;
    r.m_rho = c->m_rho; r.v_rho = c->v_rho;
    r.lr = (float)c->cfg.lr_rho;
    r.b1 = (float)c->cfg.beta1; r.b2 = (float)c->cfg.beta2; r.adam_eps = (float)c->cfg.adam_eps;
    r.ctr = c->ctr;
    r.n_x = c->cfg.n_x;
    r.pdl = c->pdl ? 1 : 0;
    return r;
}

extern "C" af_status af_ambiguity(af_ctx* c, const float* x, const float* h, float* chi) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!x || !h || !chi) FAIL(c, AF_ERR_INVALID_ARG, "af_ambiguity: NULL pointer");
    FwdArgs<float2, float> a = fwd_args(c, (const float2*)x, (const float2*)h);
    a.mode = FWD_DUMP;
    a.chi_out = (float2*)chi;
    a.cdiag = nullptr;
    CK(c, launch_fwd(c, a, c->stream));
    return AF_OK;
}

extern "C" af_status af_forward(af_ctx* c, const float* x, const float* h) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!x || !h) FAIL(c, AF_ERR_INVALID_ARG, "af_forward: x and h must not be NULL");
    CK(c, launch_fwd(c, fwd_args(c, (const float2*)x, (const float2*)h), c->stream));
    return AF_OK;
}

extern "C" af_status af_loss_grad_xh(af_ctx* c, const float* x, const float* h, double* terms, float* gx,
                                     float* gh) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (c->cfg.matched) {
        if (gh) FAIL(c, AF_ERR_INVALID_ARG, "af_loss_grad_xh: matched context: grad_h must be NULL");
        h = x;
    }
    if (!x || !h) FAIL(c, AF_ERR_INVALID_ARG, "af_loss_grad_xh: x and h must not be NULL");
    const bool want = gx != nullptr || gh != nullptr;
    CK(c, launch_eval_forward(c, (const float2*)x, (const float2*)h, c->stream, nullptr, want));
    FinArgs f = fin_args(c);
    if (!want) { f.dense_g = nullptr; f.n_dense = 0; }
    f.mode = FIN_GRAD_XH;
    f.x = (const float2*)x;
    f.h_in = (const float2*)h;
    f.terms = terms;
    f.grad_x = (float2*)gx;
    f.grad_h = (float2*)gh;
    CK(c, launch_fin(f, c->stream));
    return AF_OK;
}

extern "C" af_status af_loss_grad(af_ctx* c, const float* u, const float* h, int32_t use_hard, double* terms,
                                  float* gu, float* gh) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (c->cfg.matched && gh) FAIL(c, AF_ERR_INVALID_ARG, "af_loss_grad: matched context: grad_h must be NULL");
    if (!u || (!h && !c->cfg.matched)) FAIL(c, AF_ERR_INVALID_ARG, "af_loss_grad: u and h must not be NULL");
    const int MN = c->cfg.M * c->cfg.N;
    QuantArgs q = quant_args(c);
    float2* x = use_hard ? c->xh : c->xs;
    if (c->cfg.matched) h = (const float*)x;
    CK(c, launch_wave_from_logits(u, MN, q, use_hard ? 1 : 0, x, c->dydz, nullptr, c->stream));
    const bool want = (gu != nullptr && !use_hard) || gh != nullptr;
    CK(c, launch_eval_forward(c, x, (const float2*)h, c->stream, nullptr, want));
    FinArgs f = fin_args(c);
    if (!want) { f.dense_g = nullptr; f.n_dense = 0; }
    f.mode = use_hard ? FIN_GRAD_XH : FIN_GRAD_U;
    f.x = x;
    f.dydz = c->dydz;
    f.u = const_cast<float*>(u);
    f.h_in = (const float2*)h;
    f.terms = terms;
    f.grad_u = use_hard ? nullptr : gu;
    f.grad_h = (float2*)gh;
    CK(c, launch_fin(f, c->stream));
    return AF_OK;
}

extern "C" af_status quantize(af_ctx* c, const float* z, int64_t n, int32_t* q, float* x) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && !z)) FAIL(c, AF_ERR_INVALID_ARG, "quantize: bad z/n");
    QuantArgs qa = quant_args(c);
    CK(c, launch_quantize_z(z, n, qa, q, (float2*)x, c->stream));
    return AF_OK;
}

extern "C" af_status soft_quantize(af_ctx* c, const float* z, int64_t n, float* y, float* dydz, float* x) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && !z)) FAIL(c, AF_ERR_INVALID_ARG, "soft_quantize: bad z/n");
    QuantArgs qa = quant_args(c);
    CK(c, launch_soft_quantize_z(z, n, qa, y, dydz, (float2*)x, c->stream));
    return AF_OK;
}

extern "C" af_status af_project(af_ctx* c, float* h) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!h) FAIL(c, AF_ERR_INVALID_ARG, "af_project: h is NULL");
    CK(c, launch_project((float2*)h, c->cfg.M, c->cfg.N, c->stream));
    return AF_OK;
}

extern "C" af_status af_loss_grad_rho(af_ctx* c, const float* u, const float* h, double* terms, float* gu,
                                      float* gh, float* grho) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (c->K > 8192 || !c->rho_acc) FAIL(c, AF_ERR_INVALID_ARG, "af_loss_grad_rho: needs K <= 8192");
    if (c->cfg.matched && gh) FAIL(c, AF_ERR_INVALID_ARG, "af_loss_grad_rho: matched context: grad_h must be NULL");
    if (!u || !grho || (!h && !c->cfg.matched))
        FAIL(c, AF_ERR_INVALID_ARG, "af_loss_grad_rho: u, h and grad_rho must not be NULL");
    const int MN = c->cfg.M * c->cfg.N;
    if (c->cfg.matched) h = (const float*)c->xs;
    CK(c, launch_wave_from_logits(u, MN, quant_args(c), 0, c->xs, c->dydz, nullptr, c->stream));
    CK(c, launch_eval_forward(c, c->xs, (const float2*)h, c->stream, nullptr));
    FinArgs f = fin_args(c);
    f.mode = FIN_GRAD_U;
    f.x = c->xs; f.dydz = c->dydz;
    f.u = const_cast<float*>(u);
    f.h_in = (const float2*)h;
    f.terms = terms;
    f.grad_u = gu;
    f.grad_h = (float2*)gh;
    f.gy_out = c->gy; f.z_out = c->zb;
    CK(c, launch_fin(f, c->stream));
    RhoArgs r = rho_args(c, RHO_GRAD);
    r.grad_out = grho;
    r.pdl = 0;
    CK(c, launch_rho(r, c->stream));
    return AF_OK;
}

extern "C" af_status sqngd_attach_generator(af_ctx* c, rn_net* rn, const float* y0) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (rn && !y0) FAIL(c, AF_ERR_INVALID_ARG, "sqngd_attach_generator: y0 is NULL");
    if (rn && rn_size(rn) != c->cfg.M * c->cfg.N)
        FAIL(c, AF_ERR_INVALID_ARG, "sqngd_attach_generator: the generator has %d phases, the context M N = %d",
             rn_size(rn), c->cfg.M * c->cfg.N);
    if (rn && c->cfg.train_rho) FAIL(c, AF_ERR_INVALID_ARG, "sqngd_attach_generator: not with trained thresholds");
    CK(c, cudaStreamSynchronize(c->cap));
    c->rn = rn;
    c->rn_y0 = rn ? y0 : nullptr;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }   // the step graph changes
    return AF_OK;
}

extern "C" af_status af_get_thresholds(af_ctx* c, float* rho_host) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!rho_host) FAIL(c, AF_ERR_INVALID_ARG, "af_get_thresholds: rho is NULL");
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaStreamSynchronize(c->cap));
    CK(c, cudaMemcpy(rho_host, c->rho, sizeof(float) * c->K, cudaMemcpyDeviceToHost));
    return AF_OK;
}

extern "C" af_status af_project_thresholds(af_ctx* c, float* rho) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!rho) FAIL(c, AF_ERR_INVALID_ARG, "af_project_thresholds: rho is NULL");
    if (c->K > 8192) FAIL(c, AF_ERR_INVALID_ARG, "af_project_thresholds: needs K <= 8192");
    RhoArgs r = rho_args(c, RHO_PROJECT);
    r.rho = rho;
    r.pdl = 0;
    CK(c, launch_rho(r, c->stream));
    return AF_OK;
}

extern "C" af_status sqngd_init(af_ctx* c, const int32_t* b, const float* noise, float* u, float* h) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!b || !u || !h) FAIL(c, AF_ERR_INVALID_ARG, "sqngd_init: b, u and h must not be NULL");
    const int MN = c->cfg.M * c->cfg.N;
    CK(c, launch_init(b, (const float2*)noise, MN, c->cfg.B, c->cfg.r_n, quant_args(c), u, (float2*)h, c->stream));
    CK(c, launch_project((float2*)h, c->cfg.M, c->cfg.N, c->stream));
    return AF_OK;
}

// ------------------------------------------------------------- sqngd_step --
static bool same_state(const af_state& a, const af_state& b) {
    return a.u_dev == b.u_dev && a.h_dev == b.h_dev && a.m_u_dev == b.m_u_dev && a.v_u_dev == b.v_u_dev &&
           a.m_h_dev == b.m_h_dev && a.v_h_dev == b.v_h_dev && a.best_q_dev == b.best_q_dev &&
           a.best_h_dev == b.best_h_dev;
}

// Enqueue one outer iteration of Algorithm 1 (used for capture).
static af_status enqueue_outer(af_ctx* c, const af_state* st, cudaStream_t s) {
    const int nh = c->cfg.n_h, nx = c->cfg.n_x;
    const int MN = c->cfg.M * c->cfg.N;
    const bool matched = c->cfg.matched != 0;
    float2* h = (float2*)st->h_dev;
    bool first = true;
    if (matched) {
        // SQNAF: score the hard design with its own matched filters (best-design
        // record), then prepare the soft waveform of the first transmit step
        CK(c, launch_eval_forward(c, c->xh, c->xh, s, c->ctr));
        first = false;
        FinArgs f = fin_args(c);
        f.mode = FIN_SCORE;
        f.x = c->xh; f.h_in = c->xh;
        f.u = st->u_dev;
        f.ctr = c->ctr; f.inner = 0;
        f.log = c->log; f.eval_index = 0;
        f.snap_best = 1;
        f.best2 = c->best2; f.best_q = st->best_q_dev; f.best_h = (float2*)st->best_h_dev;
        f.next_wave = (nx > 0) ? NEXT_SOFT : NEXT_HARD;
        f.x_next = (nx > 0) ? c->xs : c->xh;
        f.dydz_next = c->dydz;
        CK(c, launch_fin(f, s));
    } else if (nh == 0) {
        CK(c, launch_wave_from_logits(st->u_dev, MN, quant_args(c), 0, c->xs, c->dydz, nullptr, s));
    }
    for (int i = 0; i < nh; ++i) {
        CK(c, launch_eval_forward(c, c->xh, h, s, first ? c->ctr : nullptr));
        first = false;
        FinArgs f = fin_args(c);
        f.mode = FIN_ADAM_H;
        f.x = c->xh; f.h_in = h; f.h = h;
        f.m_h = (float2*)st->m_h_dev; f.v_h = (float2*)st->v_h_dev;
        f.u = st->u_dev;
        f.lr = (float)c->cfg.lr_h;
        f.ctr = c->ctr; f.inner = i;
        f.log = c->log; f.eval_index = i;
        f.snap_best = (i == 0) ? 1 : 0;
        f.best2 = c->best2; f.best_q = st->best_q_dev; f.best_h = (float2*)st->best_h_dev;
        f.next_wave = (i == nh - 1) ? NEXT_SOFT : NEXT_NONE;
        f.x_next = c->xs; f.dydz_next = c->dydz;
        if (c->cfg.train_rho) f.next_wave = NEXT_NONE;      // formed below, thresholds staged
        CK(c, launch_fin(f, s));
        if (c->cfg.train_rho && i == nh - 1)
            CK(c, launch_wave_from_logits(st->u_dev, MN, quant_args(c), 0, c->xs, c->dydz, nullptr, s));
    }
    for (int j = 0; j < nx; ++j) {
        // matched: the filters are this evaluation's waveforms, which other rows
        // gather while the next waveforms are written, so the two alternate buffers
        float2* xj = (matched && (j & 1)) ? c->xs2 : c->xs;
        float2* xn = (matched && !(j & 1)) ? c->xs2 : c->xs;
        const float2* hx = matched ? xj : h;
        CK(c, launch_eval_forward(c, xj, hx, s, first ? c->ctr : nullptr));
        first = false;
        FinArgs f = fin_args(c);
        f.mode = FIN_ADAM_U;
        f.x = xj; f.dydz = c->dydz; f.h_in = hx;
        f.u = st->u_dev; f.m_u = st->m_u_dev; f.v_u = st->v_u_dev;
        f.lr = (float)c->cfg.lr_x;
        f.ctr = c->ctr; f.inner = j;
        f.log = c->log; f.eval_index = (matched ? 1 : nh) + j;
        f.next_wave = (j == nx - 1) ? NEXT_HARD : NEXT_SOFT;
        f.x_next = (j == nx - 1) ? c->xh : xn;
        f.dydz_next = c->dydz;
        if (c->rn) {
            // the generator takes the step: dL/du out of the finish kernel, then
            // Adam on theta, the forward pass to the new u and the next waveform
            f.du_out = c->du;
            const int next = f.next_wave;
            f.next_wave = NEXT_NONE;
            CK(c, launch_fin(f, s));
            CK(c, rn_enqueue_step(c->rn, c->rn_y0, c->du, st->u_dev, c->ctr, j, nx, (float)c->cfg.lr_x,
                                  (float)c->cfg.beta1, (float)c->cfg.beta2, (float)c->cfg.adam_eps, quant_args(c),
                                  next, f.x_next, c->dydz, c->pdl ? 1 : 0, s));
        } else if (c->cfg.train_rho) {
            // Adam on rho needs every element's dL/dy first: the threshold kernels
            // take the step, then the next waveform is formed with the new rho
            f.gy_out = c->gy; f.z_out = c->zb;
            RhoArgs r = rho_args(c, RHO_STEP);
            r.inner = j;
            const int next = f.next_wave;
            f.next_wave = NEXT_NONE;
            CK(c, launch_fin(f, s));
            CK(c, launch_rho(r, s));
            CK(c, launch_wave_from_logits(st->u_dev, MN, quant_args(c), next == NEXT_HARD ? 1 : 0, f.x_next,
                                          c->dydz, nullptr, s));
        } else {
            CK(c, launch_fin(f, s));
        }
    }
    return AF_OK;
}

extern "C" af_status sqngd_step(af_ctx* c, af_state* st, int32_t n_outer, double* log_host) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!st || !st->u_dev || !st->m_u_dev || !st->v_u_dev ||
        (!c->cfg.matched && (!st->h_dev || !st->m_h_dev || !st->v_h_dev)))
        FAIL(c, AF_ERR_INVALID_ARG, "sqngd_step: state buffers must not be NULL");
    if (n_outer < 0) FAIL(c, AF_ERR_INVALID_ARG, "sqngd_step: n_outer < 0");
    if (n_outer == 0) return AF_OK;
    const int ev = evals_per_outer(c);
    const int MN = c->cfg.M * c->cfg.N;

    // log capacity (the captured graph indexes the log by the device counter)
    if ((size_t)n_outer > c->log_cap_outer) {
        CK(c, cudaStreamSynchronize(c->cap));
        CK(c, cudaStreamSynchronize(c->stream));
        if (c->log) cudaFree(c->log);
        c->log = nullptr;
        size_t cap = 64;
        while (cap < (size_t)n_outer) cap *= 2;
        af_status s = dalloc(c, &c->log, cap * ev * 4);
        if (s != AF_OK) return s;
        c->log_cap_outer = cap;
        if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    }
    if (c->gexec && !same_state(c->gkey, *st)) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    if (!c->gexec) {
        cudaGraph_t g = nullptr;
        CK(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        af_status s = enqueue_outer(c, st, c->cap);
        cudaError_t e = cudaStreamEndCapture(c->cap, &g);
        if (s != AF_OK) { if (g) cudaGraphDestroy(g); return s; }
        if (e != cudaSuccess) FAIL(c, AF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { c->gexec = nullptr; FAIL(c, AF_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
        c->gkey = *st;
    }

    CK(c, cudaEventRecord(c->ev_in, c->stream));
    CK(c, cudaStreamWaitEvent(c->cap, c->ev_in, 0));
    CK(c, launch_set_counters(c->ctr, 0, st->t_h, st->t_x, st->outer, c->cap));
    if (st->best_dev) CK(c, launch_copy_f64(c->best2 + 4, st->best_dev, 4, c->cap));
    else {
        const double init[4] = {INFINITY, INFINITY, -1.0, INFINITY};
        CK(c, cudaMemcpyAsync(c->best2 + 4, init, sizeof init, cudaMemcpyHostToDevice, c->cap));
    }
    CK(c, launch_wave_from_logits(st->u_dev, MN, quant_args(c), 1, c->xh, nullptr, nullptr, c->cap));
    for (int o = 0; o < n_outer; ++o) CK(c, cudaGraphLaunch(c->gexec, c->cap));
    if (st->best_dev && (c->cfg.n_h > 0 || c->cfg.matched))
        CK(c, launch_copy_f64(st->best_dev, c->best2 + ((n_outer - 1) & 1) * 4, 4, c->cap));
    if (log_host)
        CK(c, cudaMemcpyAsync(log_host, c->log, sizeof(double) * (size_t)n_outer * ev * 4, cudaMemcpyDeviceToHost, c->cap));
    CK(c, cudaEventRecord(c->ev_out, c->cap));
    CK(c, cudaStreamWaitEvent(c->stream, c->ev_out, 0));
    st->t_h += (int64_t)n_outer * c->cfg.n_h;
    st->t_x += (int64_t)n_outer * c->cfg.n_x;
    st->outer += n_outer;
    if (log_host) return af_sync(c);
    return AF_OK;
}

// Algorithm 1's stopping test over sqngd_step (Section III-C).  After outer
// iteration t the rule fires when t - best_outer >= patience; until an
// improvement, it cannot fire before t = best_outer + patience, so the next
// chunk runs exactly up to that iteration (or to t_max).  An improvement
// inside a chunk moves the earliest firing point past the chunk's end.
extern "C" af_status sqngd_run(af_ctx* c, af_state* st, int64_t t_max, int32_t patience, af_stop* stop,
                               double* log_host, int64_t* n_done) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!st || !stop) FAIL(c, AF_ERR_INVALID_ARG, "sqngd_run: st and stop must not be NULL");
    if (patience < 1) FAIL(c, AF_ERR_INVALID_ARG, "sqngd_run: patience must be >= 1");
    if (c->cfg.n_h < 1 && !c->cfg.matched)
        FAIL(c, AF_ERR_INVALID_ARG, "sqngd_run: needs n_h >= 1 (or a matched context) to score the hard design");
    const int ev = evals_per_outer(c);
    const int64_t t0 = st->outer;
    if (n_done) *n_done = 0;
    stop->stopped = 0;
    // a fresh record counts the patience from the first iteration of this run
    if (stop->best_outer < 0) stop->best_outer = t0 - 1;
    std::vector<double> buf;
    while (st->outer < t_max) {
        const int64_t t = st->outer;   // next outer iteration
        const int64_t fire = stop->best_outer + patience;
        int64_t chunk = fire - t + 1;
        if (chunk < 1) chunk = 1;
        if (chunk > t_max - t) chunk = t_max - t;
        if (chunk > (1 << 20)) chunk = 1 << 20;
        double* lg = nullptr;
        if (log_host) lg = log_host + (size_t)(t - t0) * ev * 4;
        else {
            buf.resize((size_t)chunk * ev * 4);
            lg = buf.data();
        }
        af_status s = sqngd_step(c, st, (int32_t)chunk, lg);
        if (s != AF_OK) return s;
        if (n_done) *n_done = st->outer - t0;
        for (int64_t i = 0; i < chunk; ++i) {
            const double w = lg[(size_t)i * ev * 4 + 1];   // L_WPSL of the iteration's first (hard) evaluation
            if (w < stop->best_wpsl) { stop->best_wpsl = w; stop->best_outer = t + i; }
            if (t + i - stop->best_outer >= patience) {
                // the chunk was sized so that this is its last iteration
                stop->stopped = 1;
                return AF_OK;
            }
        }
    }
    stop->stopped = 2;
    return AF_OK;
}

extern "C" af_status af_get_rho_state(af_ctx* c, float* rho_host, float* m_host, float* v_host, int32_t* uniform) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!rho_host) FAIL(c, AF_ERR_INVALID_ARG, "af_get_rho_state: rho is NULL");
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaStreamSynchronize(c->cap));
    CK(c, cudaMemcpy(rho_host, c->rho, sizeof(float) * c->K, cudaMemcpyDeviceToHost));
    for (float* dst : {m_host, v_host}) {
        if (!dst) continue;
        const float* src = (dst == m_host) ? c->m_rho : c->v_rho;
        if (src) CK(c, cudaMemcpy(dst, src, sizeof(float) * c->K, cudaMemcpyDeviceToHost));
        else memset(dst, 0, sizeof(float) * c->K);
    }
    if (uniform) *uniform = c->rho_uniform ? 1 : 0;
    return AF_OK;
}

extern "C" af_status af_set_rho_state(af_ctx* c, const float* rho_host, const float* m_host, const float* v_host,
                                      int32_t uniform) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (!rho_host) FAIL(c, AF_ERR_INVALID_ARG, "af_set_rho_state: rho is NULL");
    if (uniform != 0 && uniform != 1) FAIL(c, AF_ERR_INVALID_ARG, "af_set_rho_state: uniform must be 0 or 1");
    if (uniform && c->cfg.train_rho) FAIL(c, AF_ERR_INVALID_ARG, "af_set_rho_state: trained thresholds read the table");
    for (int i = 0; i < c->K; ++i) {
        if (!(rho_host[i] >= 0.f && rho_host[i] <= 1.f)) FAIL(c, AF_ERR_INVALID_ARG, "rho[%d] outside [0, 1]", i);
        if (i > 0 && !(rho_host[i] >= rho_host[i - 1])) FAIL(c, AF_ERR_INVALID_ARG, "rho decreases at %d", i);
        if (uniform && rho_host[i] != (float)(((double)i + 0.5) / (double)c->K))
            FAIL(c, AF_ERR_INVALID_ARG, "af_set_rho_state: uniform = 1 but rho[%d] is not the default threshold", i);
    }
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaStreamSynchronize(c->cap));
    CK(c, cudaMemcpy(c->rho, rho_host, sizeof(float) * c->K, cudaMemcpyHostToDevice));
    if (c->m_rho && m_host) CK(c, cudaMemcpy(c->m_rho, m_host, sizeof(float) * c->K, cudaMemcpyHostToDevice));
    if (c->v_rho && v_host) CK(c, cudaMemcpy(c->v_rho, v_host, sizeof(float) * c->K, cudaMemcpyHostToDevice));
    c->rho_uniform = uniform != 0;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return AF_OK;
}

// ------------------------------------------------------------- acceptance --
extern "C" af_status af_eval_hard(af_ctx* c, const float* u, const float* h, double* out_host) {
    if (!c) return AF_ERR_INVALID_ARG;
    if (c->cfg.matched) h = nullptr;     // the filters are the hard waveforms
    if (!u || (!h && !c->cfg.matched) || !out_host) FAIL(c, AF_ERR_INVALID_ARG, "af_eval_hard: NULL pointer");
    const int M = c->cfg.M, N = c->cfg.N, MN = M * N;
    CK(c, launch_wave_hard_f64(u, (const float2*)h, MN, quant_args(c), c->level64, c->x64, c->h64, c->stream));
    FwdArgs<double2, double> a{};
    a.M = M; a.N = N; a.L = c->cfg.L; a.D = c->D; a.k_lo = c->cfg.k_lo;
    a.n_chunks = c->acc_n_chunks; a.rows_per_chunk = c->acc_rows_per_chunk;
    a.x = c->x64; a.h = c->h64; a.pre = c->pre64;
    a.tw = c->acc_fft ? c->tw64 : c->E64;
    a.wmap = c->wmap;
    a.weight_mode = c->wmap ? WM_MAP_UNWEIGHTED : WM_UNIFORM;
    a.mode = FWD_REDUCE;
    a.half_p = 0.f;
    a.pkey = c->pkey64; a.pidx = c->pidx64;
    a.cdiag = c->cdiag;
    a.fft_e = c->acc_e;
    CK(c, c->acc_fft ? launch_fwd_fft_f64(a, c->stream) : launch_fwd_dft_f64(a, c->stream));
    AccArgs g{};
    g.M = M; g.N = N; g.nblk = c->acc_nblk; g.ctas_per_pair = c->acc_ctas_per_pair;
    g.pkey = c->pkey64; g.cdiag = c->cdiag; g.x = c->x64; g.h = c->h64; g.out = c->acc_out;
    CK(c, launch_acceptance(g, c->stream));
    CK(c, cudaMemcpyAsync(out_host, c->acc_out, sizeof(double) * (4 + M), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return AF_OK;
}
