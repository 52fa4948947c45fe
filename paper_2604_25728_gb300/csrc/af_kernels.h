// af_kernels.h -- launch interfaces shared by the translation units of the
// library (host side).  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace af {

// How a forward pass scores each cell.
enum WeightMode : int {
    WM_UNIFORM = 0,     // key = |chi|^2 (the uniform weight is applied afterwards)
    WM_MAP = 1,         // key = w^2 |chi|^2, cells with w <= 0 skipped
    WM_MAP_UNWEIGHTED = 2  // key = |chi|^2 on cells with w > 0 (acceptance PSL)
};

enum FwdMode : int {
    FWD_REDUCE = 0,     // per-CTA max/argmax (+ p-norm partials), chi never stored
    FWD_DUMP = 1        // write chi to chi_out [M][M][D][L]
};

// Arguments of the fused forward pass (product + Doppler transform +
// sidelobe reduction).  C is float2 or double2, K the key type.
template <typename C, typename K>
struct FwdArgs {
    int M, N, L, D, k_lo;
    int n_chunks;          // delay chunks per pair; grid = M*M*n_chunks
    int rows_per_chunk;    // multiple of the row slots per CTA
    const C* x;            // [M][N] transmit waveforms (not Doppler-modulated)
    const C* h;            // [M][N] receive filters
    const C* pre;          // [N] e^{j 2 pi nu_0 n} (FFT grid) -- unused by the DFT path
    const C* tw;           // FFT twiddle tables (FFT path) / [N][L] phasor table (DFT path)
    const float* wmap;     // [D][L] ROI weights or nullptr
    int weight_mode;       // WeightMode
    int mode;              // FwdMode
    float half_p;          // p/2 for the p-norm partials, 0 = exact max only
    K* pkey;               // [grid] best key per CTA (-1 = none)
    long long* pidx;       // [grid] its linear cell index
    float* pvmax;          // [grid] p-norm partial: max key
    float* psum;           // [grid] p-norm partial: sum (key/max)^(p/2)
    double2* cdiag;        // [M] chi_mm(0,0) = sum_n x_m conj(h_m), FP64 (may be nullptr)
    C* chi_out;            // FWD_DUMP output
    long long* ctr_inc;    // if set, CTA 0 adds 1 to ctr_inc[0] (outer-iteration counter)
    int fft_e;             // FFT path: values per thread (8, 16 or 32); selects the twiddle plan
    int fft_nt;            // FFT path: threads per CTA (256, or 512 for FP32 rows of >= 1024 bins); 0 = 256
    C* pchi;               // [grid] chi at each CTA's best cell (may be nullptr)
    int pdl;               // launch with programmatic stream serialisation
};

// Dense adjoint of the p-norm sidelobe loss on the FFT grid.  The grid spans
// only the winning class: `grid` CTAs, chunk b mod cpp_cls[c] of pair
// b / cpp_cls[c] of class c.
struct AdjArgs {
    int M, N, L, D, k_lo;
    int grid;              // CTAs of the launch (the same for either winning class)
    int cpp_cls[2];        // delay chunks per pair when the auto (0) / cross (1) class wins
    int rows_cls[2];       // delays per chunk (a multiple of the row slots)
    int rpc_max;           // the larger of the two (sizes the h window)
    int nt;                // threads per CTA (256, or 512 for rows of >= 1024 bins)
    int* cls_buf;          // the winning class, written by CTA 0 for the summing kernel
    const float2* x;       // [M][N] waveforms of this evaluation
    const float2* h;       // [M][N] filters
    const float2* pre;     // [N] e^{j 2 pi nu_0 n}
    const float2* tw;      // FFT twiddle tables
    const float* wmap;     // [D][L] or nullptr
    int weight_mode;
    float w0;
    double eps;
    float half_p;          // p/2
    int nblk_fwd, ctas_per_pair_fwd;
    const float* pvmax;    // forward p-norm partials
    const float* psum;
    float2* part;          // [grid][2][N] per-CTA partial rows (grad x_m, grad h_l)
    float2* dense;         // [2][M][N] summed sidelobe gradient (x, h)
    int fft_e;
    int pdl;
};
struct AdjGeom {
    int grid, cpp[2], rows[2], rpc_max;
};
cudaError_t launch_adj(const AdjArgs& a, cudaStream_t s);
cudaError_t adj_prepare(int L, int N, int E, int NT, int rpc);
int adj_smem_bytes(int L, int N, int E, int NT, int rpc);
int adj_threads(int L, int E);
void adj_geometry(int M, int D, int L, int E, int NT, int slots, AdjGeom* g);

// FFT path with E values per thread: dynamic shared memory bytes (-1 if L
// unsupported), row slots per 256-thread CTA, and the default E for L.
// Shared memory of one forward CTA of NT threads whose delay chunk holds rpc
// rows (rpc <= 0: one row per slot); -1 if the shape is not built.
int fft_smem_bytes(int L, int N, bool fp64, int E, int NT = 256, int rpc = 0);
int fft_rows_per_cta(int L, int E, int NT = 256);
int fft_default_elems(int L, bool fp64);
int fft_default_threads(int L, int E, bool fp64);
int fft_occupancy(int L, int N, int E, bool fp64, int NT, int rpc);   // resident CTAs per SM (reduce kernel)
cudaError_t launch_fwd_fft_f32(const FwdArgs<float2, float>& a, cudaStream_t s);
cudaError_t launch_fwd_fft_f64(const FwdArgs<double2, double>& a, cudaStream_t s);
cudaError_t fft_prepare_f32(int L, int N, int E, int NT, int rpc);
cudaError_t fft_prepare_f64(int L, int N, int E, int NT, int rpc);

// Raise the dynamic shared-memory limit of the DFT kernels a context will use.
cudaError_t dft_prepare_f32(int N);
cudaError_t dft_prepare_f64(int N);

// Direct DFT path (any grid), SIMT; a single bin (L = 1) runs as a
// cross-correlation kernel with its own delays per CTA.
int dft_rows_per_cta(int L);
int dft_col_tiles(int L);
cudaError_t launch_fwd_dft_f32(const FwdArgs<float2, float>& a, cudaStream_t s);
cudaError_t launch_fwd_dft_f64(const FwdArgs<double2, double>& a, cudaStream_t s);

// Narrow-window path on tcgen05 tensor cores: one CTA per 128 delays of
// `tiles` pairs and per column tile of LB bins (LB a power of two in 16..128,
// at most gemm_bins_per_tile(L));
// BF16 hi/lo split operands, FP32 accumulation in tensor memory.
constexpr int kGemmRows = 128;      // delays per tile (MMA M)
struct GemmArgs {
    FwdArgs<float2, float> f;   // x, h, wmap, mode, pkey/pidx/pchi, cdiag, chi_out, ctr_inc, pdl
    const void* bimg;           // [M][n_ct][n_kc][hi | lo][2 LB x 2 spc] BF16 images of B_m = x_m E
    int* err;                   // bit 1 set when a pipeline wait timed out
    int lb;                     // bins per column tile (16, 32, 64 or 128)
    int n_ct;                   // column tiles = ceil(L / LB)
    int n_kc;                   // sample chunks = ceil(N / spc)
    int spc;                    // samples per pipeline stage
    int sb, sa;                 // stages of B images (shared memory) and of lag products (tensor memory)
    int tiles;                  // pairs (delay tiles) per CTA sharing each B stage (1, or 2 when M*M is even)
    unsigned long long timeout_ns;  // limit of every pipeline wait
    int test_stall;             // failure-detection test: the MMA issuer waits on a barrier nothing completes
    // Split schedule (0 CTAs: one CTA per tile).  split_ctas CTAs each take an
    // equal contiguous range of the split_work sample chunks of all tiles in
    // tile order; a tile shared by several CTAs is finished by the last of
    // them to arrive (tile_cnt), which adds the pieces' FP32 partials (part,
    // [tile][max_pieces][2 LB columns][128 rows]) in piece order.
    int split_ctas;
    long long split_work;
    int max_pieces;
    float* part;
    int* tile_cnt;              // [tiles], zeroed by the B-image kernel of each evaluation
};
// Sample chunks of delay block b (128 delays from k_lo + 128 b): the chunks
// c0 .. c0 + count - 1 of spc samples hold every sample n with a valid lag
// product n + k in [0, N) for some delay of the block.
__host__ __device__ inline int gemm_block_chunks(int k_lo, int D, int N, int spc, int b, int* c0) {
    const int d0 = b * kGemmRows;
    const int k_first = k_lo + d0;
    const int k_last = k_lo + (D < d0 + kGemmRows ? D : d0 + kGemmRows) - 1;
    const int n_begin = k_last < 0 ? -k_last : 0;
    const int n_end = N < N - k_first ? N : N - k_first;
    *c0 = n_begin / spc;
    return (n_end + spc - 1) / spc - *c0;
}
// A split schedule over `ctas` CTAs for P pairs x n_blocks delay blocks x
// n_ct column tiles (one pair per CTA): ok when every CTA gets at least one
// chunk and at most kGemmMaxSeg pieces; work = total chunks, max_pieces =
// most CTAs sharing one tile.
constexpr int kGemmMaxSeg = 8;
struct GemmSplitPlan { bool ok; long long work; int max_pieces; int max_segs; };
GemmSplitPlan gemm_split_plan(int P, int n_blocks, int n_ct, int k_lo, int D, int N, int spc, int ctas);
int gemm_bins_per_tile(int L);
int gemm_smem_bytes(int LB, int N, int spc, int sb, int sa, int tiles);
int gemm_ctas_per_sm(int LB, int N, int spc, int sb, int sa, int tiles);   // CTAs that fit on one SM
bool gemm_shape_supported(int LB, int N, int spc, int sb, int sa, int tiles);
cudaError_t gemm_prepare(int LB, int N, int spc, int sb, int sa, int tiles);
cudaError_t launch_fwd_gemm(const GemmArgs& g, cudaStream_t s);
// B_m = x_m(n) e^{j 2 pi nu_j n} images of one evaluation (E: [N][L] FP32 phasors)
cudaError_t launch_gemm_bimg(const float2* x, const float2* E, int M, int N, int L, int LB, int spc, void* img,
                             int* tile_cnt, int n_tiles, int pdl, cudaStream_t s);
size_t gemm_bimg_bytes(int M, int N, int L, int LB, int spc);

// Record the message of a failed call that has no context (read back by
// af_last_error(NULL) on the same thread).
void set_thread_error(const char* msg);

struct QuantArgs;
struct FinArgs;
struct AccArgs;
struct RhoArgs;
}  // namespace af
struct rn_net;
namespace af {
cudaError_t rn_enqueue_step(rn_net* n, const float* y0, const float* du, float* u, const long long* ctr, int inner,
                            int n_x, float lr, float b1, float b2, float eps, const QuantArgs& q, int next_wave,
                            float2* x_next, float* dydz_next, int pdl, cudaStream_t s);
int rn_size(const rn_net* n);
int rho_smem_bytes(int K);
cudaError_t rho_prepare(int K);
cudaError_t launch_rho(const RhoArgs& a, cudaStream_t s);
cudaError_t launch_wave_from_logits(const float* u, int n, const QuantArgs& q, int hard, float2* x,
                                    float* dydz, int32_t* qout, cudaStream_t s);
cudaError_t launch_quantize_z(const float* z, long long n, const QuantArgs& q, int32_t* qout, float2* x,
                              cudaStream_t s);
cudaError_t launch_soft_quantize_z(const float* z, long long n, const QuantArgs& q, float* y, float* dydz,
                                   float2* x, cudaStream_t s);
cudaError_t launch_wave_hard_f64(const float* u, const float2* h, int n, const QuantArgs& q,
                                 const double2* level64, double2* x64, double2* h64, cudaStream_t s);
cudaError_t launch_fin(const FinArgs& a, cudaStream_t s);
cudaError_t launch_project(float2* h, int M, int N, cudaStream_t s);
cudaError_t launch_init(const int32_t* b, const float2* noise, int n, int B, int r_n, const QuantArgs& q,
                        float* u, float2* h, cudaStream_t s);
cudaError_t launch_acceptance(const AccArgs& a, cudaStream_t s);
cudaError_t launch_set_counters(long long* ctr, long long a0, long long a1, long long a2, long long a3,
                                cudaStream_t s);
cudaError_t launch_copy_f64(double* dst, const double* src, int n, cudaStream_t s);

}  // namespace af
