// af_gemm.cu -- forward pass on a narrow Doppler window as a tensor-core
// contraction (sm_103a, tcgen05 + tensor memory).
//
// chi[(pair, d), j] = sum_n conj(h_l(n+k)) [x_m(n) e^{j 2 pi nu_j n}]
// (Eq. 6 restated per row): a product A B with A[(pair, d), n] =
// conj(h_l(n + k)) -- a Hankel matrix of the filter, the same for every
// transmit waveform -- and B_m[n, j] = x_m(n) E[n, j], E[n, j] = e^{j 2 pi nu_j n},
// one image per transmit waveform, built for each evaluation by
// gemm_bimg_kernel from x and the FP64-built phasor table.  Complex arithmetic
// is embedded in a real GEMM: the K index interleaves (Re A(n), Im A(n)) and
// the output columns interleave (Re chi_j, Im chi_j), so with b = B_m[n, j]
// B[(n,0),(j,0)] = Re b, B[(n,1),(j,0)] = -Im b, B[(n,0),(j,1)] = Im b,
// B[(n,1),(j,1)] = Re b.
//
// Precision: both operands are split into BF16 pairs v = hi + lo and the
// product is taken as Ah Bh + Ah Bl + Al Bh (the lo*lo term is below FP32
// accumulation noise), accumulating in FP32 in tensor memory.
//
// One CTA owns 128 consecutive delays of one pair (the MMA M) and LB bins
// (N = 2 LB columns).  Roles:
//   warps 0-3  copy their row's split filter samples (thread = row = TMEM
//              lane; the CTA splits its window of conj(h_l) into BF16 hi/lo
//              once) for a chunk of 32 samples into a tensor-memory A stage
//              (tcgen05.st); afterwards they read the accumulator back
//              (tcgen05.ld) and run the sidelobe reduction.
//   warp 4     allocates tensor memory; lane 0 issues the MMAs.
//   warp 5     lane 0 streams the pair's B_m image (hi | lo, in the canonical
//              no-swizzle K-major layout) with cp.async.bulk.
// Stages are double-buffered with mbarriers; every wait is bounded and a
// timeout sets bit 1 of the error flag and ends the kernel cleanly.
//
// With fewer tiles than SMs a second instantiation runs the split schedule:
// the CTAs that fit at once each take an equal range of the sample chunks of
// all tiles, cut into pieces at tile boundaries, and a tile shared by several
// CTAs is finished by the last of them to arrive (an atomic ticket; no CTA
// waits for another), which adds the pieces' FP32 partials in piece order.
#include <cuda_bf16.h>

#include <vector>

#include "af_common.cuh"
#include "af_kernels.h"
#include "af_tc.cuh"

namespace af {

constexpr int kTM = kGemmRows;             // 128 delays per tile

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`.  Gives up when another role has
// aborted (unless `drain`) or after `limit_ns`, which aborts the CTA.  The
// abort flag and the clock are looked at every 64 polls only.
__device__ __noinline__ bool gwait_slow(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                        bool drain, unsigned long long limit_ns) {
    const unsigned long long t0 = gtimer();
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (tc::mbar_try_wait(bar, parity)) return true;
        if (!drain && *abort_flag) return false;
        if (gtimer() - t0 > limit_ns) {
            *abort_flag = 1;
            if (err) atomicOr(err, 2);
            return false;
        }
    }
}
__device__ __forceinline__ bool gwait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                      bool drain, unsigned long long limit_ns) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    return gwait_slow(bar, parity, abort_flag, err, drain, limit_ns);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);   // .x in the low half
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo_f(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi_f(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

template <int NR> __device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t (&r)[NR]);
template <> __device__ __forceinline__ void tmem_st<16>(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
template <> __device__ __forceinline__ void tmem_st<32>(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
          "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
          "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D[tmem] (+)= A[tmem] * B[smem]: A from tensor memory (lane = row, K pairs per column).
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(d_tmem), "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ bool gbetter(float a, long long ia, float b, long long ib) {
    return a > b || (a == b && ia < ib);
}

// Tensor-memory columns of a CTA: T accumulators of NC columns plus SA A
// stages of T tiles x (SPC hi + SPC lo) columns, rounded up to a power of
// two (0 if more than 512).
__host__ __device__ constexpr int gemm_tmem_cols(int NC, int SPC, int SA, int T) {
    return (T * NC + 2 * SPC * SA * T <= 128) ? 128 : (T * NC + 2 * SPC * SA * T <= 256) ? 256
         : (T * NC + 2 * SPC * SA * T <= 512) ? 512 : 0;
}

// One piece of a CTA's work: chunks ib .. ib + nch - 1 of tile q (pair group
// pg, column tile ct, delay block blk), whose window starts at chunk c0 of the
// samples.  whole: the piece is the whole tile; else it is piece `piece` of
// the `npieces` CTAs that share the tile.
struct GSeg {
    int q, pg, ct, blk, c0, ib, nch, piece, npieces, whole;
};

// kSB stages of B images in shared memory (filled by bulk copies), kSA
// stages of lag products in tensor memory (filled by tcgen05.st); the CTA's
// chunk g (counted over all its pieces) uses B stage g % kSB and A stage
// g % kSA.
template <int NC, int kSPC, int kSB, int kSA, int T, bool SPLIT>
__global__ void __launch_bounds__(32 * (4 * T + 2), 1)
fwd_gemm_kernel(const GemmArgs g) {
    const FwdArgs<float2, float>& a = g.f;
    constexpr int kKC = 2 * kSPC;                    // real K per chunk
    constexpr int LB = NC / 2;
    constexpr int NPROD = kTM * T;                   // producer / epilogue threads
    constexpr int WMMA = 4 * T, WLOAD = 4 * T + 1;   // MMA and loader warps
    constexpr int STAGE_BYTES = NC * kKC * 2 * 2;    // hi | lo images
    constexpr int TCOLS = gemm_tmem_cols(NC, kSPC, kSA, T);
    static_assert(NC % 32 == 0 && NC >= 32 && NC <= 256, "column tile");
    static_assert(TCOLS > 0 && kSPC % 8 == 0, "stage shape");
    static_assert(!SPLIT || T == 1, "the split schedule takes one pair per CTA");

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* bst = smem_raw;                                        // [kSB][STAGE_BYTES]
    const int XH = kSPC * g.n_kc + kTM;                                   // per tile: split conj(h) window
    uint2* xh_base = reinterpret_cast<uint2*>(smem_raw + kSB * STAGE_BYTES);

    __shared__ __align__(8) uint64_t bfull[kSB], bempty[kSB], afull[kSA], aempty[kSA], accfull, never;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ float rk[T][4];
    __shared__ long long ri[T][4];
    __shared__ float2 rc[T][4];
    __shared__ DFloat red[T][2][4];
    __shared__ GSeg s_seg[kGemmMaxSeg];
    __shared__ int s_nseg, s_ticket;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int bx = blockIdx.x;
    const int P = a.M * a.M;
    const int PG = P / T;
    const int PGC = PG * g.n_ct;
    const int N = a.N, L = a.L, D = a.D;

    if (tid == 0) {
        for (int s = 0; s < kSB; ++s) {
            tc::mbar_init(&bfull[s], 1);
            tc::mbar_init(&bempty[s], 1);   // one MMA commit
        }
        for (int s = 0; s < kSA; ++s) {
            tc::mbar_init(&afull[s], NPROD / 32);   // one arrival per producer warp
            tc::mbar_init(&aempty[s], 1);
        }
        tc::mbar_init(&accfull, 1);
        tc::mbar_init(&never, 1);          // nothing arrives here (failure-detection test)
        s_abort = 0;
        tc::mbar_fence_init();
        // This CTA's pieces of work.  Tiles are ordered pair-group-fastest:
        // consecutive tiles share the delay block and column tile -- hence every
        // B image, which their CTAs read from L2.
        int ns = 0;
        if constexpr (!SPLIT) {
            GSeg sg;
            sg.q = bx;
            sg.pg = bx % PG;
            sg.ct = (bx / PG) % g.n_ct;
            sg.blk = bx / PGC;
            sg.nch = gemm_block_chunks(a.k_lo, D, N, kSPC, sg.blk, &sg.c0);
            sg.ib = 0; sg.piece = 0; sg.npieces = 1; sg.whole = 1;
            s_seg[ns++] = sg;
        } else {
            // chunks [w0, w1) of all tiles' chunks in tile order
            const long long W = g.split_work, G = g.split_ctas;
            const long long w0 = (long long)bx * W / G, w1 = (long long)(bx + 1) * W / G;
            long long base = 0;                       // first chunk of block b
            int b = 0, c0b = 0;
            int nb = gemm_block_chunks(a.k_lo, D, N, kSPC, 0, &c0b);
            for (long long x = w0; x < w1 && ns < kGemmMaxSeg;) {
                while (x >= base + (long long)PGC * nb) {
                    base += (long long)PGC * nb;
                    ++b;
                    nb = gemm_block_chunks(a.k_lo, D, N, kSPC, b, &c0b);
                }
                const int qi = (int)((x - base) / nb);        // tile within the block
                const long long ts = base + (long long)qi * nb, te = ts + nb;
                const long long xe = w1 < te ? w1 : te;
                GSeg sg;
                sg.q = b * PGC + qi;
                sg.pg = qi % PG;
                sg.ct = qi / PG;
                sg.blk = b;
                sg.c0 = c0b;
                sg.ib = (int)(x - ts);
                sg.nch = (int)(xe - x);
                // the CTAs holding the tile's first and last chunks
                const long long cf = ((ts + 1) * G - 1) / W, cl = (te * G - 1) / W;
                sg.piece = (int)(bx - cf);
                sg.npieces = (int)(cl - cf + 1);
                sg.whole = sg.npieces == 1;
                s_seg[ns++] = sg;
                x = xe;
            }
        }
        s_nseg = ns;
    }
    if (warp == WMMA) {
        __syncwarp();
        tc::tmem_alloc(&s_tmem, TCOLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = s_tmem;
    const int nseg = SPLIT ? s_nseg : 1;
    volatile int* abort_flag = &s_abort;
    int total = 0;                                    // chunks of this CTA
    for (int k = 0; k < nseg; ++k) total += s_seg[k].nch;

    if (warp == WLOAD) {
        // ---------------------------------------------------- B loader --
        // Stage s of chunk g: one bulk copy of the whole stage, completing on bfull[s].
        // The T pairs of a CTA share their transmit waveform (T divides M), so one B_m image.
        int issued = 0;
        // the B_m images are written by the kernel just ahead in the stream
        pdl_wait();
        pdl_trigger();
        if (lane == 0) {
            bool okl = true;
            int gi = 0;
            for (int k = 0; okl && k < nseg; ++k) {
                const GSeg sg = s_seg[k];
                const int m_cta = (sg.pg * T) / a.M;
                const unsigned char* img = reinterpret_cast<const unsigned char*>(g.bimg) +
                    (((size_t)m_cta * g.n_ct + sg.ct) * g.n_kc + sg.c0 + sg.ib) * (size_t)STAGE_BYTES;
                for (int i = 0; i < sg.nch; ++i, ++gi) {
                    const int s = gi % kSB;
                    // the MMAs have finished with stage s
                    if (gi >= kSB &&
                        !gwait(&bempty[s], ((gi / kSB) - 1) & 1, abort_flag, g.err, false, g.timeout_ns)) {
                        okl = false;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(&bfull[s], STAGE_BYTES);
                    tc::bulk_g2s(bst + s * STAGE_BYTES, img + (size_t)i * STAGE_BYTES, STAGE_BYTES, &bfull[s]);
                    issued = gi + 1;
                }
            }
            // every stage in flight has landed, and every MMA commit has
            // arrived, before the CTA exits
            for (int i = max(0, issued - kSB); i < issued; ++i)
                gwait(&bfull[i % kSB], (i / kSB) & 1, abort_flag, g.err, true, g.timeout_ns);
            for (int i = max(0, total - kSB); i < total; ++i)
                gwait(&bempty[i % kSB], (i / kSB) & 1, abort_flag, g.err, true, g.timeout_ns);
        }
    } else if (warp == WMMA) {
        // ------------------------------------------------- MMA issuer --
        pdl_wait();
        pdl_trigger();
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16(kTM, NC);
            // Descriptors of stage 0; a stage, a K step and the lo image are
            // constant offsets in the start-address field (address >> 4,
            // bits 0-13), so the issue loop is a few adds per MMA.
            const uint64_t dbase = tc::smem_desc(tc::smem_u32(bst), 128, (kKC / 8) * 128);
            // failure-detection test: wait on a barrier nothing completes; the
            // bounded wait gives up, aborts the CTA and reports a timeout
            bool go = true;
            if (g.test_stall) go = gwait(&never, 0, abort_flag, g.err, false, g.timeout_ns);
            constexpr uint64_t kStageStep = STAGE_BYTES >> 4, kLoStep = (NC * kKC * 2) >> 4, kKStep = 256 >> 4;
            int gi = 0, commits = 0;
            for (int k = 0; go && k < nseg; ++k) {
                const int nchk = s_seg[k].nch;
                for (int i = 0; i < nchk; ++i, ++gi) {
                    const int s = gi % kSB, sa = gi % kSA;
                    if (!gwait(&bfull[s], (gi / kSB) & 1, abort_flag, g.err, false, g.timeout_ns) ||
                        !gwait(&afull[sa], (gi / kSA) & 1, abort_flag, g.err, false, g.timeout_ns)) {
                        go = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint64_t dh = dbase + (uint64_t)s * kStageStep;
                    const uint64_t dl = dh + kLoStep;
                    const uint32_t acc0 = (i > 0) ? 1u : 0u;    // each piece starts a fresh accumulator
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        const uint32_t d_t = tbase + t * NC;
                        const uint32_t a_hi = tbase + T * NC + (sa * T + t) * kKC;
#pragma unroll
                        for (int q = 0; q < kKC / 16; ++q) {
                            mma_ts(d_t, a_hi + 8 * q, dh + q * kKStep, idesc, q == 0 ? acc0 : 1u);
                            mma_ts(d_t, a_hi + 8 * q, dl + q * kKStep, idesc, 1u);
                            mma_ts(d_t, a_hi + kSPC + 8 * q, dh + q * kKStep, idesc, 1u);
                        }
                    }
                    tc::mma_commit(&bempty[s]);
                    tc::mma_commit(&aempty[sa]);
                }
                // the piece's accumulator is complete (after an abort: every
                // MMA issued so far has finished)
                tc::mma_commit(&accfull);
                ++commits;
            }
            if (commits > 0) gwait(&accfull, (commits - 1) & 1, abort_flag, g.err, true, g.timeout_ns);
        }
    } else {
        // ------------------------------------ producers and epilogue --
        pdl_wait();
        pdl_trigger();
        if (a.ctr_inc != nullptr && bx == 0 && tid == 0) a.ctr_inc[0] += 1;
        const int t = tid / kTM, r = tid % kTM;          // this thread's tile and row
        const int wq = warp & 3;                          // lane quarter of tensor memory
        const uint32_t trow = tbase + ((uint32_t)(wq * 32) << 16);
        uint2* hs = xh_base + t * XH;                    // [kSPC * n_kc + kTM] split conj(h_l) window
        bool ok = true;
        int gi = 0;
        for (int k = 0; k < nseg; ++k) {
        const GSeg sg = s_seg[k];
        const int pair = sg.pg * T + t;
        const int m = pair / a.M, l = pair - m * a.M;
        const int ob = (pair * a.n_chunks + sg.blk) * g.n_ct + sg.ct;   // partial record (pair-major)
        const int d0 = sg.blk * kTM;
        const int k_first = a.k_lo + d0;
        const int c0 = sg.c0 + sg.ib, nch = sg.nch;
        const float2* xm = a.x + (size_t)m * N;
        const float2* hl = a.h + (size_t)l * N;
        const int nh = kSPC * nch + kTM;
        // the previous piece's copies have read the window
        if (k > 0) asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory");
        // the window conj(h_l(p)), p = SPC c0 + k_first + i, split once into
        // BF16 (re, im) hi and lo pairs: all loads of a batch are in flight
        // before the first store
        constexpr int FB = 8;
        for (int i0 = r; i0 < nh; i0 += kTM * FB) {
            float2 hv[FB];
#pragma unroll
            for (int q = 0; q < FB; ++q) {
                const int i = i0 + q * kTM;
                const int p = kSPC * c0 + k_first + i;
                hv[q] = (i < nh && p >= 0 && p < N) ? hl[p] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < FB; ++q) {
                const int i = i0 + q * kTM;
                const float re = hv[q].x, im = -hv[q].y;
                const uint32_t ph = pack_bf16(re, im);
                if (i < nh) hs[i] = make_uint2(ph, pack_bf16(re - bf16_lo_f(ph), im - bf16_hi_f(ph)));
            }
        }
        // chi_mm(0, 0) = sum_n x_m(n) conj(h_m(n)) (SNRL, Eq. 38) while the first
        // B stages are still in flight, by the CTA holding the first chunk of
        // delay block 0: exact products, double-float partials and tree
        if (a.cdiag != nullptr && sg.blk == 0 && sg.ct == 0 && sg.ib == 0) {
            const bool diag = (m == l);
            DFloat sr = {0.f, 0.f}, si = {0.f, 0.f};
            if (diag) {
                for (int n0 = r; n0 < N; n0 += kTM * FB) {
                    float2 xv[FB], hv[FB];
#pragma unroll
                    for (int q = 0; q < FB; ++q) {
                        const int n = n0 + q * kTM;
                        xv[q] = n < N ? xm[n] : make_float2(0.f, 0.f);
                        hv[q] = n < N ? hl[n] : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int q = 0; q < FB; ++q) df_acc_xconjh(xv[q], hv[q], sr, si);
                }
            }
            const DFloat dr = df_warp_sum(sr), di = df_warp_sum(si);
            if (lane == 0) { red[t][0][warp & 3] = dr; red[t][1][warp & 3] = di; }
            asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory");
            if (diag && r == 0) {
                DFloat tr = red[t][0][0], ti = red[t][1][0];
                for (int w = 1; w < 4; ++w) { tr = df_add(tr, red[t][0][w]); ti = df_add(ti, red[t][1][w]); }
                a.cdiag[m] = make_double2(df_to_double(tr), df_to_double(ti));
            }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory");

        for (int i = 0; i < nch; ++i, ++gi) {
            const int s = gi % kSA;
            if (ok && gi >= kSA) {
                // one lane polls; the warp takes its verdict before the
                // aligned tensor-memory stores
                bool w = true;
                if (lane == 0) w = gwait(&aempty[s], ((gi / kSA) - 1) & 1, abort_flag, g.err, false, g.timeout_ns);
                if (!__shfl_sync(0xffffffffu, w, 0)) ok = false;
                tc::fence_after_sync();
            }
            if (!ok) continue;
            // row r, sample n = SPC (c0 + i) + u: conj(h_l(n + k)) = hs[SPC i + r + u]
            uint32_t hi[kSPC], lo[kSPC];
            const uint2* hc = hs + i * kSPC + r;
#pragma unroll
            for (int u = 0; u < kSPC; ++u) {
                const uint2 hv = hc[u];
                hi[u] = hv.x;
                lo[u] = hv.y;
            }
            const uint32_t acol = trow + T * NC + (s * T + t) * kKC;
            tmem_st<kSPC>(acol, hi);
            tmem_st<kSPC>(acol + kSPC, lo);
            tmem_st_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&afull[s])) : "memory");
        }

        // ---- epilogue: accumulator -> sidelobe reduction (Eqs. 7-9) ----
        float best = -1.f;
        long long best_idx = 0x7fffffffffffffffLL;
        float2 best_c = make_float2(0.f, 0.f);
        bool acc_ready = ok;
        if (lane == 0 && ok) acc_ready = gwait(&accfull, k & 1, abort_flag, g.err, false, g.timeout_ns);
        acc_ready = __shfl_sync(0xffffffffu, acc_ready, 0);
        if (acc_ready) tc::fence_after_sync();
        // A shared tile: every piece stores its partial ([column][row], so a
        // warp's stores are contiguous) and takes a ticket; the last piece to
        // arrive adds all partials in piece order (the same sum whichever CTA
        // is last) and finishes the tile.  No CTA waits for another.
        bool finish = true;
        const size_t pstride = (size_t)NC * kTM;
        const float* tile_part = SPLIT ? g.part + (size_t)sg.q * g.max_pieces * pstride : nullptr;
        if (SPLIT && !sg.whole) {
            if (acc_ready) {
                float* mine = g.part + ((size_t)sg.q * g.max_pieces + sg.piece) * pstride + r;
#pragma unroll 1
                for (int cc = 0; cc < NC / 32; ++cc) {
                    float v[32];
                    tc::tmem_ld32(trow + t * NC + cc * 32, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int b = 0; b < 32; ++b) __stcg(mine + (size_t)(cc * 32 + b) * kTM, v[b]);
                }
                __threadfence();
            }
            asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory");
            if (tid == 0) s_ticket = atomicAdd(g.tile_cnt + sg.q, 1);
            asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory");
            finish = s_ticket == sg.npieces - 1;
            if (finish) __threadfence();
        }
        if (finish && acc_ready) {
            const int d = d0 + r;
            const int kd = a.k_lo + d;
            const bool row_ok = d < D && !(m == l && kd == 0);
            const bool dump = a.mode == FWD_DUMP;
            const bool fast = !dump && a.weight_mode == WM_UNIFORM;
#pragma unroll 1
            for (int cc = 0; cc < NC / 32; ++cc) {
                float v[32];
                tc::tmem_ld32(trow + t * NC + cc * 32, v);
                tc::tmem_ld_wait();
                if (SPLIT && !sg.whole) {
                    float acc[32];
#pragma unroll
                    for (int b = 0; b < 32; ++b) acc[b] = 0.f;
                    for (int pc = 0; pc < sg.npieces; ++pc) {
                        if (pc == sg.piece) {
#pragma unroll
                            for (int b = 0; b < 32; ++b) acc[b] += v[b];
                        } else {
                            const float* src = tile_part + pc * pstride + (size_t)(cc * 32) * kTM + r;
#pragma unroll
                            for (int b = 0; b < 32; ++b) acc[b] += __ldcg(src + (size_t)b * kTM);
                        }
                    }
#pragma unroll
                    for (int b = 0; b < 32; ++b) v[b] = acc[b];
                }
                if (fast) {
                    // cells of a row are visited in increasing index order, so
                    // a group only matters if its largest key beats the best so
                    // far, and then its first maximal cell is the candidate
                    float key[16];
                    const int jb = sg.ct * LB + cc * 16;
#pragma unroll
                    for (int b = 0; b < 16; ++b)
                        key[b] = (row_ok && jb + b < L) ? fmaf(v[2 * b], v[2 * b], v[2 * b + 1] * v[2 * b + 1]) : -1.f;
                    float gm = key[0];
#pragma unroll
                    for (int b = 1; b < 16; ++b) gm = fmaxf(gm, key[b]);
                    if (gm > best) {
                        int bsel = 15;
                        float cx = v[30], cy = v[31];
#pragma unroll
                        for (int b = 14; b >= 0; --b)
                            if (key[b] == gm) { bsel = b; cx = v[2 * b]; cy = v[2 * b + 1]; }
                        best = gm;
                        best_idx = ((long long)pair * D + d) * L + jb + bsel;
                        best_c = make_float2(cx, cy);
                    }
                    continue;
                }
#pragma unroll
                for (int b = 0; b < 16; ++b) {
                    const int jj = sg.ct * LB + cc * 16 + b;
                    const float re = v[2 * b], im = v[2 * b + 1];
                    if (dump) {
                        if (d < D && jj < L) a.chi_out[((size_t)pair * D + d) * L + jj] = make_float2(re, im);
                        continue;
                    }
                    if (!row_ok || jj >= L) continue;
                    float key = re * re + im * im;
                    if (a.weight_mode != WM_UNIFORM) {
                        const float w = __ldg(a.wmap + (size_t)d * L + jj);
                        key = (w > 0.f) ? (a.weight_mode == WM_MAP ? w * w * key : key) : -1.f;
                    }
                    const long long cell = ((long long)pair * D + d) * L + jj;
                    if (gbetter(key, cell, best, best_idx)) { best = key; best_idx = cell; best_c = make_float2(re, im); }
                }
            }
        }
        tc::fence_before_sync();
        if (finish && a.mode != FWD_DUMP) {
            for (int o = 16; o > 0; o >>= 1) {
                const float obk = __shfl_xor_sync(0xffffffffu, best, o);
                const long long oi = __shfl_xor_sync(0xffffffffu, best_idx, o);
                const float ocx = __shfl_xor_sync(0xffffffffu, best_c.x, o);
                const float ocy = __shfl_xor_sync(0xffffffffu, best_c.y, o);
                if (gbetter(obk, oi, best, best_idx)) { best = obk; best_idx = oi; best_c = make_float2(ocx, ocy); }
            }
            if (lane == 0) { rk[t][wq] = best; ri[t][wq] = best_idx; rc[t][wq] = best_c; }
            asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory");
            if (r == 0) {
                float b = rk[t][0];
                long long bi = ri[t][0];
                float2 bc = rc[t][0];
                for (int w = 1; w < 4; ++w)
                    if (gbetter(rk[t][w], ri[t][w], b, bi)) { b = rk[t][w]; bi = ri[t][w]; bc = rc[t][w]; }
                a.pkey[ob] = b;
                a.pidx[ob] = (b >= 0.f) ? bi : -1;
                if (a.pchi) a.pchi[ob] = bc;
                if (a.pvmax) { a.pvmax[ob] = 0.f; a.psum[ob] = 0.f; }
            }
        }
        }  // pieces
    }

    tc::fence_before_sync();
    __syncthreads();
    if (warp == WMMA) {
        __syncwarp();
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, TCOLS);
    }
}

// B_m images of one evaluation (see the top of this file): thread (m, ct, c,
// jj, g) writes, for bin j = ct LB + jj and samples n = c SPC + 4 g .. + 3,
// the two 16-byte core-matrix rows (u = 0, 1) of the hi and of the lo image.
// Row u = 0 holds (Re b, -Im b) per sample, row u = 1 (Im b, Re b), with
// b = x_m(n) E[n, j] in FP32 (E built in FP64 on the host); bins beyond L and
// samples beyond N are zero.
// It also zeroes the split schedule's tile counters for the contraction that
// follows (the previous contraction has finished: this kernel waits for the
// kernel ahead of it, which waited for that contraction).
__global__ void gemm_bimg_kernel(const float2* __restrict__ x, const float2* __restrict__ E, int M, int N, int L,
                                 int LB, int n_ct, int n_kc, int spc, uint16_t* __restrict__ img,
                                 int* __restrict__ tile_cnt, int n_tiles) {
    pdl_wait();
    pdl_trigger();
    const int G = spc / 4;
    const long long total = (long long)M * n_ct * n_kc * LB * G;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tile_cnt != nullptr && id < n_tiles) tile_cnt[id] = 0;
    if (id >= total) return;
    const int jj = (int)(id % LB);
    long long rest = id / LB;
    const int g = (int)(rest % G); rest /= G;
    const int c = (int)(rest % n_kc); rest /= n_kc;
    const int ct = (int)(rest % n_ct);
    const int m = (int)(rest / n_ct);
    const int j = ct * LB + jj;
    const int NC = 2 * LB, KC = 2 * spc;
    float re[4], im[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int n = c * spc + 4 * g + q;
        float2 b = make_float2(0.f, 0.f);
        if (n < N && j < L) b = cmul(x[(size_t)m * N + n], E[(size_t)n * L + j]);
        re[q] = b.x;
        im[q] = b.y;
    }
    uint16_t* hi_img = img + ((((size_t)m * n_ct + ct) * n_kc + c) * 2) * (size_t)NC * KC;
    uint16_t* lo_img = hi_img + (size_t)NC * KC;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        uint32_t h4[4], l4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float v0 = (u == 0) ? re[q] : im[q];    // K index 2 s    (Re A)
            const float v1 = (u == 0) ? -im[q] : re[q];   // K index 2 s + 1 (Im A)
            const uint32_t ph = pack_bf16(v0, v1);
            h4[q] = ph;
            l4[q] = pack_bf16(v0 - bf16_lo_f(ph), v1 - bf16_hi_f(ph));
        }
        const int ci = 2 * jj + u;
        // core matrix (ci / 8, g) of 8 x 8 BF16, row ci % 8: 16 contiguous bytes
        const size_t off = (size_t)(ci / 8) * (KC / 8) * 64 + (size_t)g * 64 + (ci % 8) * 8;
        *reinterpret_cast<uint4*>(hi_img + off) = make_uint4(h4[0], h4[1], h4[2], h4[3]);
        *reinterpret_cast<uint4*>(lo_img + off) = make_uint4(l4[0], l4[1], l4[2], l4[3]);
    }
}

cudaError_t launch_gemm_bimg(const float2* x, const float2* E, int M, int N, int L, int LB, int spc, void* img,
                             int* tile_cnt, int n_tiles, int pdl, cudaStream_t s) {
    const int n_ct = (L + LB - 1) / LB, n_kc = (N + spc - 1) / spc;
    if (spc % 4 != 0 || n_tiles < 0) return cudaErrorInvalidValue;
    long long total = (long long)M * n_ct * n_kc * LB * (spc / 4);
    if (tile_cnt != nullptr && total < n_tiles) total = n_tiles;
    const int threads = 256;
    const long long blocks = (total + threads - 1) / threads;
    return launch_ex(gemm_bimg_kernel, dim3((unsigned)blocks), dim3(threads), 0, s, pdl != 0, x, E, M, N, L, LB,
                     n_ct, n_kc, spc, reinterpret_cast<uint16_t*>(img), tile_cnt, n_tiles);
}

// The split schedule of the CTAs (see GemmArgs), checked by walking it as the
// kernel does: every CTA must get at least one chunk (else a tile could wait
// for a piece that no CTA holds) and at most kGemmMaxSeg pieces.
GemmSplitPlan gemm_split_plan(int P, int n_blocks, int n_ct, int k_lo, int D, int N, int spc, int ctas) {
    GemmSplitPlan plan{false, 0, 0, 0};
    if (P < 1 || n_blocks < 1 || n_ct < 1 || spc < 1 || ctas < 1) return plan;
    const long long PGC = (long long)P * n_ct;
    std::vector<int> nb(n_blocks);
    long long W = 0;
    for (int b = 0; b < n_blocks; ++b) {
        int c0 = 0;
        nb[b] = gemm_block_chunks(k_lo, D, N, spc, b, &c0);
        if (nb[b] < 1) return plan;
        W += PGC * nb[b];
    }
    if (W < ctas) return plan;
    const long long G = ctas;
    int max_pieces = 1, max_segs = 0;
    for (long long c = 0; c < G; ++c) {
        const long long w0 = c * W / G, w1 = (c + 1) * W / G;
        long long base = 0;
        int b = 0, segs = 0;
        for (long long x = w0; x < w1;) {
            while (x >= base + PGC * nb[b]) { base += PGC * nb[b]; ++b; }
            const long long qi = (x - base) / nb[b];
            const long long ts = base + qi * nb[b], te = ts + nb[b];
            const long long cf = ((ts + 1) * G - 1) / W, cl = (te * G - 1) / W;
            if (cl - cf + 1 > max_pieces) max_pieces = (int)(cl - cf + 1);
            ++segs;
            x = w1 < te ? w1 : te;
        }
        if (segs > max_segs) max_segs = segs;
    }
    plan.ok = max_segs >= 1 && max_segs <= kGemmMaxSeg;
    plan.work = W;
    plan.max_pieces = max_pieces;
    plan.max_segs = max_segs;
    return plan;
}

size_t gemm_bimg_bytes(int M, int N, int L, int LB, int spc) {
    const size_t n_ct = (L + LB - 1) / LB, n_kc = (N + spc - 1) / spc;
    return (size_t)M * n_ct * n_kc * 2 * (size_t)(2 * LB) * (2 * spc) * sizeof(uint16_t);
}

// The widest column tile: the smallest power of two >= L, from 16 to 128 bins.
int gemm_bins_per_tile(int L) {
    int lb = 16;
    while (lb < L && lb < 128) lb <<= 1;
    return lb;
}

// Dynamic shared memory of a CTA (0 if the shape does not fit).  It is padded
// so that the CTAs that fit on an SM never ask for more tensor memory than the
// SM's 512 columns, so no allocation has to wait.
int gemm_smem_bytes(int LB, int N, int spc, int sb, int sa, int tiles) {
    const int NC = 2 * LB;
    if (!(LB == 16 || LB == 32 || LB == 64 || LB == 128)) return 0;
    const int tcols = gemm_tmem_cols(NC, spc, sa, tiles);
    if (tcols == 0 || spc <= 0 || tiles < 1) return 0;
    const int n_kc = (N + spc - 1) / spc;
    const int need = sb * NC * spc * 8 + tiles * (int)sizeof(uint2) * (spc * n_kc + kTM);
    const int floor_bytes = 228 * 1024 / (512 / tcols + 1) + 1024;
    const int b = need > floor_bytes ? need : floor_bytes;
    return b <= 227 * 1024 ? b : 0;
}

// CTAs that fit on one SM at once: tensor memory (512 columns) and shared
// memory (228 KB, 1 KB of it reserved per CTA) decide.
int gemm_ctas_per_sm(int LB, int N, int spc, int sb, int sa, int tiles) {
    const int smem = gemm_smem_bytes(LB, N, spc, sb, sa, tiles);
    const int tcols = gemm_tmem_cols(2 * LB, spc, sa, tiles);
    if (smem <= 0 || tcols <= 0) return 1;
    const int by_tmem = 512 / tcols, by_smem = (228 * 1024) / (smem + 1024);
    const int n = by_tmem < by_smem ? by_tmem : by_smem;
    return n > 0 ? n : 1;
}

template <int NC, int SPC, int SB, int SA, int T>
static cudaError_t launch_cfg(const GemmArgs& g, int smem, cudaStream_t s, bool prepare_only) {
    if constexpr (gemm_tmem_cols(NC, SPC, SA, T) == 0) {
        return cudaErrorInvalidValue;   // more tensor memory than an SM has
    } else {
    // the split schedule is built for one pair per CTA in the default pipeline shape
    constexpr bool kCanSplit = (T == 1 && SPC == 32 && SB == 2 && SA == 2);
    if (g.split_ctas > 0 && !kCanSplit) return cudaErrorInvalidValue;
    void (*kern)(const GemmArgs) = fwd_gemm_kernel<NC, SPC, SB, SA, T, false>;
    if constexpr (kCanSplit) {
        if (prepare_only) {
            cudaError_t e = set_smem_once(reinterpret_cast<const void*>(fwd_gemm_kernel<NC, SPC, SB, SA, T, true>), smem);
            if (e != cudaSuccess) return e;
        }
        if (g.split_ctas > 0) kern = fwd_gemm_kernel<NC, SPC, SB, SA, T, true>;
    }
    cudaError_t e = set_smem_once(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess || prepare_only) return e;
    const int grid = g.split_ctas > 0 ? g.split_ctas : g.f.M * g.f.M / T * g.f.n_chunks * g.n_ct;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * (4 * T + 2));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    int na = 0;
    if (g.f.pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, g);
    }
}

// Pipeline shapes built: samples per stage x B stages x A stages.
#define AF_GEMM_SHAPES(X) X(32, 2, 2) X(32, 4, 2) X(16, 4, 2) X(16, 8, 4)

template <int NC, int T>
static cudaError_t launch_nct(const GemmArgs& g, int smem, cudaStream_t s, bool prepare_only) {
#define AF_GEMM_CASE(P, B, A) \
    if (g.spc == P && g.sb == B && g.sa == A) return launch_cfg<NC, P, B, A, T>(g, smem, s, prepare_only);
    AF_GEMM_SHAPES(AF_GEMM_CASE)
#undef AF_GEMM_CASE
    return cudaErrorInvalidValue;
}

template <int NC>
static cudaError_t launch_nc(const GemmArgs& g, int smem, cudaStream_t s, bool prepare_only) {
    return g.tiles == 2 ? launch_nct<NC, 2>(g, smem, s, prepare_only) : launch_nct<NC, 1>(g, smem, s, prepare_only);
}

bool gemm_shape_supported(int LB, int N, int spc, int sb, int sa, int tiles) {
    bool listed = false;
#define AF_GEMM_LISTED(P, B, A) listed = listed || (spc == P && sb == B && sa == A);
    AF_GEMM_SHAPES(AF_GEMM_LISTED)
#undef AF_GEMM_LISTED
    return listed && (tiles == 1 || tiles == 2) && gemm_smem_bytes(LB, N, spc, sb, sa, tiles) > 0;
}

static cudaError_t dispatch(const GemmArgs& g, cudaStream_t s, bool prepare_only) {
    if (!gemm_shape_supported(g.lb, g.f.N, g.spc, g.sb, g.sa, g.tiles)) return cudaErrorInvalidValue;
    const int smem = gemm_smem_bytes(g.lb, g.f.N, g.spc, g.sb, g.sa, g.tiles);
    switch (2 * g.lb) {
        case 32: return launch_nc<32>(g, smem, s, prepare_only);
        case 64: return launch_nc<64>(g, smem, s, prepare_only);
        case 128: return launch_nc<128>(g, smem, s, prepare_only);
        case 256: return launch_nc<256>(g, smem, s, prepare_only);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t gemm_prepare(int LB, int N, int spc, int sb, int sa, int tiles) {
    GemmArgs g{};
    g.lb = LB;
    g.f.N = N;
    g.spc = spc;
    g.sb = sb;
    g.sa = sa;
    g.tiles = tiles;
    return dispatch(g, nullptr, true);
}

cudaError_t launch_fwd_gemm(const GemmArgs& g, cudaStream_t s) {
    if (g.f.n_chunks * kTM < g.f.D || g.spc <= 0 || g.n_kc * g.spc < g.f.N || g.timeout_ns == 0 ||
        g.n_ct * g.lb < g.f.L)
        return cudaErrorInvalidValue;
    const int P = g.f.M * g.f.M;
    if (!(g.tiles == 1 || g.tiles == 2) || P % g.tiles != 0) return cudaErrorInvalidValue;
    if (g.split_ctas > 0 && (g.tiles != 1 || g.part == nullptr || g.tile_cnt == nullptr || g.max_pieces < 1 ||
                             g.split_work < g.split_ctas))
        return cudaErrorInvalidValue;
    return dispatch(g, s, false);
}

}  // namespace af
