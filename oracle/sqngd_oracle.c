/*
 * sqngd_oracle.c -- plain FP64 CPU oracle for the SQNGD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check in __graft_entry__ and the CPU-baseline leg of bench.py may load it.
 * It shares no code, header, table or constant generator with the CUDA path;
 * neither side includes or links the other.
 *
 * Paper: "Joint Design of Doppler-Resilient Unimodular Discrete-Phase
 * Waveforms and Receiving Filters for MIMO Radars" (SQNGD).  Every function
 * names the equation or section it follows.  Readings where the paper is
 * silent or ambiguous are marked READING and are the same ones the design
 * notes list:
 *   - sample index n runs 0..N-1 (Eq. 6 counts from 1; that multiplies chi by
 *     a unimodular factor and changes no |chi| and no loss),
 *   - Doppler nu is in cycles per chip (the paper's f/N),
 *   - the auto-AF term excludes every tau = 0 cell (Eq. 8, literal),
 *   - the max in Eqs. 7-9 is differentiated at one cell: the larger value,
 *     ties broken towards the smaller linear cell index; WAPSL wins a tie
 *     against WCPSL,
 *   - thresholds rho_i = (i + 1/2)/K, a_i = 1/(2B), K = B*r_n (Eq. 24 with
 *     the worked example Eq. 25),
 *   - the hard quantizer is the c -> infinity limit of Eq. 43:
 *     q = #{i : rho_i <= z}, level q/B, phase index b = q mod B,
 *   - Adam uses beta1 = 0.9, beta2 = 0.999, eps = 1e-8 unless told otherwise.
 *
 * Parity status: every function below is pinned by the CPU test suite
 * (closed forms, library routines, invariants, finite differences and the
 * paper's worked example), except the multi-iteration optimisation loop as a
 * whole, whose trajectory is chaotic: "parity unpinned" for full-run design
 * quality (the per-step pieces are pinned individually).
 *
 * Layouts (all row-major, complex numbers as interleaved re,im doubles):
 *   x, h          [M][N]            waveform-major (Eq. 16, vec of N x M)
 *   chi           [M][M][D][L]      pair (m, l) = (transmit m, filter l),
 *                                   d = k - k_lo, j = Doppler bin
 *   weights       [D][L] or NULL    NULL means w = 1/N on every ROI cell
 *   linear cell   ((m*M + l)*D + d)*L + j
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

/* e^{j 2 pi t} for t in cycles; the integer part is removed first so the
 * argument of cos/sin stays in [0, 2 pi). */
static cplx phasor(double t)
{
    double f = t - floor(t);
    return cos(TWO_PI * f) + I * sin(TWO_PI * f);
}

/* ------------------------------------------------------------------------ */
/* Eq. 6: chi_ml(k, nu) = sum_n x_m(n) conj(h_l(n + k)) e^{j 2 pi nu n},      */
/* with h_l(p) = 0 outside 0 <= p < N.                                      */
/* ------------------------------------------------------------------------ */
static cplx af_cell(int N, const cplx* xm, const cplx* hl, int k, double nu)
{
    cplx s = 0.0;
    for (int n = 0; n < N; ++n) {
        int p = n + k;
        if (p < 0 || p >= N) continue;
        s += xm[n] * conj(hl[p]) * phasor(nu * (double)n);
    }
    return s;
}

/* The same sum with the phasors e^{j 2 pi nu n} of one Doppler bin taken
 * from a table row e[n] = phasor(nu n) (built once per call). */
static cplx af_cell_tab(int N, const cplx* xm, const cplx* hl, int k, const cplx* e)
{
    cplx s = 0.0;
    for (int n = 0; n < N; ++n) {
        int p = n + k;
        if (p < 0 || p >= N) continue;
        s += xm[n] * conj(hl[p]) * e[n];
    }
    return s;
}

/* Table E[j][n] = phasor(nu_j n). */
static cplx* phasor_table(int N, int L, const double* nu)
{
    cplx* e = (cplx*)malloc(sizeof(cplx) * (size_t)N * L);
    for (int j = 0; j < L; ++j)
        for (int n = 0; n < N; ++n) e[(size_t)j * N + n] = phasor(nu[j] * (double)n);
    return e;
}

void or_ambiguity(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                  const double* x_ri, const double* h_ri, double* chi_ri)
{
    const cplx* x = (const cplx*)x_ri;
    const cplx* h = (const cplx*)h_ri;
    cplx* chi = (cplx*)chi_ri;
    int D = k_hi - k_lo + 1;
    long long rows = (long long)M * M * D;
    cplx* E = phasor_table(N, L, nu);
#pragma omp parallel for schedule(dynamic, 4)
    for (long long r = 0; r < rows; ++r) {
        int d = (int)(r % D);
        int pair = (int)(r / D);
        int m = pair / M, l = pair % M;
        for (int j = 0; j < L; ++j)
            chi[r * L + j] = af_cell_tab(N, x + (size_t)m * N, h + (size_t)l * N,
                                         k_lo + d, E + (size_t)j * N);
    }
    free(E);
}

/* Individual cells, for checking very large grids at sampled points. */
void or_ambiguity_cells(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                        const double* x_ri, const double* h_ri,
                        int ncell, const long long* cells, double* out_ri)
{
    const cplx* x = (const cplx*)x_ri;
    const cplx* h = (const cplx*)h_ri;
    cplx* out = (cplx*)out_ri;
    int D = k_hi - k_lo + 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int c = 0; c < ncell; ++c) {
        long long id = cells[c];
        int j = (int)(id % L);
        int d = (int)((id / L) % D);
        int pair = (int)(id / ((long long)L * D));
        int m = pair / M, l = pair % M;
        out[c] = af_cell(N, x + (size_t)m * N, h + (size_t)l * N, k_lo + d, nu[j]);
    }
    (void)M;
}

/* ------------------------------------------------------------------------ */
/* Loss: Eqs. 7-9 (WPSL), Eq. 37 (L_WPSL), Eq. 38 (p_m), Eq. 39 (p_tar),      */
/* Eq. 41 (L_SNRL), Eq. 42 (total).                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int M, N, L, k_lo, k_hi;
    const double* nu;
    const double* w;     /* [D][L] or NULL */
    double eps, snrl_db, pnorm;
} or_cfg;

static double cell_weight(const or_cfg* c, int d, int j)
{
    return c->w ? c->w[(size_t)d * c->L + j] : 1.0 / (double)c->N;
}

/* Whether a cell belongs to the ROI of the auto (cls = 0) or cross (cls = 1)
 * term.  Eq. 8 takes m1 = m2 and tau != 0; Eq. 9 takes m1 != m2, every tau. */
static int cell_class(int m, int l, int k)
{
    if (m == l) return (k == 0) ? -1 : 0;
    return 1;
}

/* Per-class result of the sidelobe scan. */
typedef struct {
    double vmax;        /* max of w|chi| */
    long long arg;      /* linear cell index of the max (lowest index on ties) */
    double psum;        /* sum of (w|chi| / vmax)^p, p-norm variant only */
    int any;
} or_peak;

static void scan_af(const or_cfg* c, const cplx* x, const cplx* h, or_peak pk[2])
{
    int M = c->M, N = c->N, L = c->L, D = c->k_hi - c->k_lo + 1;
    long long rows = (long long)M * M * D;
    for (int cls = 0; cls < 2; ++cls) { pk[cls].vmax = 0; pk[cls].arg = -1; pk[cls].psum = 0; pk[cls].any = 0; }
    cplx* E = phasor_table(N, L, c->nu);
    /* pass 1: max and argmax of w|chi| per class */
    double* rowmax = (double*)malloc(sizeof(double) * rows);
    long long* rowarg = (long long*)malloc(sizeof(long long) * rows);
#pragma omp parallel for schedule(dynamic, 4)
    for (long long r = 0; r < rows; ++r) {
        int d = (int)(r % D), pair = (int)(r / D), m = pair / M, l = pair % M;
        int k = c->k_lo + d;
        rowmax[r] = -1.0; rowarg[r] = -1;
        if (cell_class(m, l, k) < 0) continue;
        for (int j = 0; j < L; ++j) {
            double w = cell_weight(c, d, j);
            if (w <= 0) continue;
            double v = w * cabs(af_cell_tab(N, x + (size_t)m * N, h + (size_t)l * N, k, E + (size_t)j * N));
            if (v > rowmax[r]) { rowmax[r] = v; rowarg[r] = r * L + j; }
        }
    }
    for (long long r = 0; r < rows; ++r) {
        int d = (int)(r % D), pair = (int)(r / D), m = pair / M, l = pair % M;
        int cls = cell_class(m, l, c->k_lo + d);
        if (cls < 0 || rowarg[r] < 0) continue;
        /* rows are visited in increasing index, so '>' keeps the lowest index on ties */
        if (!pk[cls].any || rowmax[r] > pk[cls].vmax) {
            pk[cls].vmax = rowmax[r]; pk[cls].arg = rowarg[r]; pk[cls].any = 1;
        }
    }
    /* pass 2 (p-norm variant): sum of (v / vmax)^p per class */
    if (c->pnorm > 0) {
        double* rowsum = (double*)calloc((size_t)rows, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
        for (long long r = 0; r < rows; ++r) {
            int d = (int)(r % D), pair = (int)(r / D), m = pair / M, l = pair % M;
            int k = c->k_lo + d;
            int cls = cell_class(m, l, k);
            if (cls < 0 || pk[cls].vmax <= 0) continue;
            double s = 0;
            for (int j = 0; j < L; ++j) {
                double w = cell_weight(c, d, j);
                if (w <= 0) continue;
                double v = w * cabs(af_cell_tab(N, x + (size_t)m * N, h + (size_t)l * N, k, E + (size_t)j * N));
                s += pow(v / pk[cls].vmax, c->pnorm);
            }
            rowsum[r] = s;
        }
        for (long long r = 0; r < rows; ++r) {
            int d = (int)(r % D), pair = (int)(r / D), m = pair / M, l = pair % M;
            int cls = cell_class(m, l, c->k_lo + d);
            if (cls >= 0) pk[cls].psum += rowsum[r];
        }
        free(rowsum);
    }
    free(rowmax); free(rowarg); free(E);
}

/* The class value that enters Eq. 37: the peak itself (exact max, the
 * paper's loss) or the p-norm (sum v^p)^(1/p) (smooth extension). */
static double class_value(const or_cfg* c, const or_peak* p)
{
    if (!p->any) return 0.0;
    if (c->pnorm > 0) return p->vmax * pow(p->psum, 1.0 / c->pnorm);
    return p->vmax;
}

/* terms[0] = L, terms[1] = L_WPSL, terms[2] = WAPSL, terms[3] = WCPSL,
 * terms[4] = L_SNRL, terms[5] = winning class (0 auto, 1 cross).
 * p[m] = p_m of Eq. 38.  cells[0], cells[1] = argmax cell of the auto and
 * cross class (-1 if the class is empty).  Returns 0. */
static void loss_core(const or_cfg* c, const cplx* x, const cplx* h,
                      double* terms, double* p, long long* cells, or_peak pk[2])
{
    int M = c->M, N = c->N;
    scan_af(c, x, h, pk);
    double wapsl = class_value(c, &pk[0]);
    double wcpsl = class_value(c, &pk[1]);
    double lw = (wapsl >= wcpsl) ? wapsl : wcpsl;                    /* Eq. 37 */
    double ptar = pow(10.0, -c->snrl_db / 20.0);                     /* Eq. 39 */
    double ls = 0;
    for (int m = 0; m < M; ++m) {
        cplx a00 = 0;                                                 /* h_m^H x_m */
        for (int n = 0; n < N; ++n) a00 += conj(h[(size_t)m * N + n]) * x[(size_t)m * N + n];
        double pm = cabs(a00) / (double)N;                           /* Eq. 38 */
        if (p) p[m] = pm;
        ls += (pm - ptar) * (pm - ptar);
    }
    ls /= (double)M;                                                  /* Eq. 41 */
    if (terms) {
        terms[0] = c->eps * lw + (1.0 - c->eps) * ls;                 /* Eq. 42 */
        terms[1] = lw; terms[2] = wapsl; terms[3] = wcpsl; terms[4] = ls;
        terms[5] = (wapsl >= wcpsl) ? 0.0 : 1.0;
    }
    if (cells) { cells[0] = pk[0].arg; cells[1] = pk[1].arg; }
}

void or_loss(int M, int N, int L, const double* nu, int k_lo, int k_hi,
             const double* w, double eps, double snrl_db, double pnorm,
             const double* x_ri, const double* h_ri,
             double* terms, double* p, long long* cells)
{
    or_cfg c = { M, N, L, k_lo, k_hi, nu, w, eps, snrl_db, pnorm };
    or_peak pk[2];
    loss_core(&c, (const cplx*)x_ri, (const cplx*)h_ri, terms, p, cells, pk);
}

/* ------------------------------------------------------------------------ */
/* Analytic gradient of Eq. 42 w.r.t. x and h, in the real-pair convention  */
/* grad = dL/dRe + j dL/dIm (the receive filter is the pair H_Re, H_Im of    */
/* Eq. 28).  For a real function of chi with G = dL/dRe chi + j dL/dIm chi:  */
/*   grad x_m(n)  += G * h_l(n+k) * e^{-j 2 pi nu n}                         */
/*   grad h_l(p)  += conj(G) * x_m(p-k) * e^{+j 2 pi nu (p-k)}               */
/* because chi is linear in x_m(n) with coefficient conj(h_l(n+k)) e^{..}   */
/* and linear in conj(h_l(p)) with coefficient x_m(p-k) e^{..}.             */
/* For |chi|, G = chi / |chi|.                                               */
/* ------------------------------------------------------------------------ */
static void add_cell_grad(const or_cfg* c, const cplx* x, const cplx* h,
                          long long cell, cplx G, cplx* gx, cplx* gh)
{
    int M = c->M, N = c->N, L = c->L, D = c->k_hi - c->k_lo + 1;
    int j = (int)(cell % L);
    int d = (int)((cell / L) % D);
    int pair = (int)(cell / ((long long)L * D));
    int m = pair / M, l = pair % M, k = c->k_lo + d;
    double nu = c->nu[j];
    for (int n = 0; n < N; ++n) {
        int p = n + k;
        if (p < 0 || p >= N) continue;
        cplx e = phasor(nu * (double)n);
        gx[(size_t)m * N + n] += G * h[(size_t)l * N + p] * conj(e);
        gh[(size_t)l * N + p] += conj(G) * x[(size_t)m * N + n] * e;
    }
}

/* use_cell: NULL => differentiate the max at the oracle's own argmax; else
 * the cell whose value is taken as the WPSL (for comparing against another
 * evaluator that picked a different one of near-tied cells).  Exact-max
 * variant only; the p-norm variant has a unique gradient. */
void or_grad_xh(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                const double* w, double eps, double snrl_db, double pnorm,
                const double* x_ri, const double* h_ri, const long long* use_cell,
                double* terms, double* gx_ri, double* gh_ri)
{
    or_cfg c = { M, N, L, k_lo, k_hi, nu, w, eps, snrl_db, pnorm };
    const cplx* x = (const cplx*)x_ri;
    const cplx* h = (const cplx*)h_ri;
    cplx* gx = (cplx*)gx_ri;
    cplx* gh = (cplx*)gh_ri;
    int D = k_hi - k_lo + 1;
    double t[6];
    double* p = (double*)malloc(sizeof(double) * M);
    long long cells[2];
    or_peak pk[2];
    loss_core(&c, x, h, t, p, cells, pk);
    if (terms) memcpy(terms, t, sizeof t);
    memset(gx, 0, sizeof(cplx) * (size_t)M * N);
    memset(gh, 0, sizeof(cplx) * (size_t)M * N);
    int cls = (int)t[5];

    if (pnorm <= 0) {
        long long cell = use_cell ? *use_cell : cells[cls];
        if (cell >= 0) {
            int j = (int)(cell % L), d = (int)((cell / L) % D);
            int pair = (int)(cell / ((long long)L * D));
            cplx a = af_cell(N, x + (size_t)(pair / M) * N, h + (size_t)(pair % M) * N,
                             k_lo + d, nu[j]);
            double mag = cabs(a);
            if (mag > 0) add_cell_grad(&c, x, h, cell, eps * cell_weight(&c, d, j) * a / mag, gx, gh);
        }
    } else if (pk[cls].any && pk[cls].vmax > 0) {
        /* d/dv_c (sum v^p)^(1/p) = (v_c / V)^(p-1), V the class p-norm.  Every
         * cell of the winning class adds G = eps w (w|chi|/V)^(p-1) chi/|chi|
         * through the two adjoint sums above (as add_cell_grad, with the
         * phasors from a table).  Rows are split over threads with private
         * accumulators, summed in thread order afterwards. */
        double V = class_value(&c, &pk[cls]);
        long long rows = (long long)M * M * D;
        cplx* E = phasor_table(N, L, nu);
        int nt = 1;
#ifdef _OPENMP
        nt = omp_get_max_threads();
#endif
        cplx* acc = (cplx*)calloc((size_t)nt * 2 * M * N, sizeof(cplx));
#pragma omp parallel num_threads(nt)
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            cplx* tgx = acc + (size_t)tid * 2 * M * N;
            cplx* tgh = tgx + (size_t)M * N;
#pragma omp for schedule(static)
            for (long long r = 0; r < rows; ++r) {
                int d = (int)(r % D), pair = (int)(r / D), m = pair / M, l = pair % M;
                int k = k_lo + d;
                if (cell_class(m, l, k) != cls) continue;
                for (int j = 0; j < L; ++j) {
                    double wt = cell_weight(&c, d, j);
                    if (wt <= 0) continue;
                    const cplx* e = E + (size_t)j * N;
                    cplx a = af_cell_tab(N, x + (size_t)m * N, h + (size_t)l * N, k, e);
                    double mag = cabs(a);
                    if (mag <= 0) continue;
                    cplx G = eps * pow(wt * mag / V, pnorm - 1.0) * wt * a / mag;
                    for (int n = 0; n < N; ++n) {
                        int q = n + k;
                        if (q < 0 || q >= N) continue;
                        tgx[(size_t)m * N + n] += G * h[(size_t)l * N + q] * conj(e[n]);
                        tgh[(size_t)l * N + q] += conj(G) * x[(size_t)m * N + n] * e[n];
                    }
                }
            }
        }
        for (int t = 0; t < nt; ++t)
            for (size_t i = 0; i < (size_t)M * N; ++i) {
                gx[i] += acc[(size_t)t * 2 * M * N + i];
                gh[i] += acc[(size_t)t * 2 * M * N + (size_t)M * N + i];
            }
        free(acc);
        free(E);
    }
    /* SNRL term: L_SNRL = (1/M) sum (p_m - p_tar)^2, p_m = |A_mm(0,0)|/N with
     * A_mm(0,0) = sum_n x_m(n) conj(h_m(n)) (Eq. 38, nu = 0, tau = 0). */
    double ptar = pow(10.0, -snrl_db / 20.0);
    for (int m = 0; m < M; ++m) {
        cplx a00 = 0;
        for (int n = 0; n < N; ++n) a00 += x[(size_t)m * N + n] * conj(h[(size_t)m * N + n]);
        double mag = cabs(a00);
        if (mag <= 0) continue;
        cplx G = (1.0 - eps) * (2.0 / M) * (p[m] - ptar) / (double)N * a00 / mag;
        for (int n = 0; n < N; ++n) {
            gx[(size_t)m * N + n] += G * h[(size_t)m * N + n];
            gh[(size_t)m * N + n] += conj(G) * x[(size_t)m * N + n];
        }
    }
    free(p);
}

/* ------------------------------------------------------------------------ */
/* Soft quantization with copies, Eq. 24:                                   */
/*   Q_A(z) = sum_{i<K} a_i [tanh(c (z - rho_i)) + 1]                        */
/* and its derivative sum a_i c (1 - tanh^2).                                */
/* ------------------------------------------------------------------------ */
void or_soft_quantize(int n, const double* z, int K, const double* rho,
                      double a, double c, double* y, double* dydz)
{
#pragma omp parallel for schedule(static)
    for (int e = 0; e < n; ++e) {
        double s = 0, ds = 0;
        for (int i = 0; i < K; ++i) {
            double t = tanh(c * (z[e] - rho[i]));
            s += a * (t + 1.0);
            ds += a * c * (1.0 - t * t);
        }
        y[e] = s;
        if (dydz) dydz[e] = ds;
    }
}

/* The literal piecewise hard quantizer of Eq. 43 at finite c, for checking
 * the c -> infinity reading against the paper's worked example. */
void or_hard_quantize_literal(int n, const double* z, int K, const double* rho,
                              double a, double c, double* y)
{
    for (int e = 0; e < n; ++e) {
        double v;
        if (z[e] < rho[0]) v = 0.0;
        else if (z[e] >= rho[K - 1]) v = 2.0 * a * K;
        else {
            int i = 0;
            while (!(rho[i] <= z[e] && z[e] < rho[i + 1])) ++i;
            double mid = 0.5 * (rho[i] + rho[i + 1]);
            or_soft_quantize(1, &mid, K, rho, a, c, &v, NULL);
        }
        y[e] = v;
    }
}

/* READING of Eq. 43 (c -> infinity): q = #{i : rho_i <= z}; the normalised
 * level is q / B and the transmitted phase index b = q mod B (Eq. 5). */
void or_hard_quantize(int n, const double* z, int K, const double* rho, int B,
                      int* q, int* b)
{
    for (int e = 0; e < n; ++e) {
        int cnt = 0;
        for (int i = 0; i < K; ++i)
            if (rho[i] <= z[e]) ++cnt;
        q[e] = cnt;
        if (b) b[e] = cnt % B;
    }
}

/* Thresholds and coefficients of Eq. 24, READING rho_i = (i + 1/2)/K,
 * a = 1/(2B). */
void or_thresholds(int B, int r_n, double* rho, double* a)
{
    int K = B * r_n;
    for (int i = 0; i < K; ++i) rho[i] = ((double)i + 0.5) / (double)K;
    if (a) *a = 1.0 / (2.0 * B);
}

/* ------------------------------------------------------------------------ */
/* Energy projection, Eq. 32: h_m <- sqrt(N / ||h_m||^2) h_m.                 */
/* ------------------------------------------------------------------------ */
void or_project(int M, int N, double* h_ri)
{
    cplx* h = (cplx*)h_ri;
    for (int m = 0; m < M; ++m) {
        double e = 0;
        for (int n = 0; n < N; ++n) { double a = cabs(h[(size_t)m * N + n]); e += a * a; }
        if (e <= 0) continue;
        double s = sqrt((double)N / e);
        for (int n = 0; n < N; ++n) h[(size_t)m * N + n] *= s;
    }
}

/* ------------------------------------------------------------------------ */
/* Adam (Section III-A/III-C: Adam on H_Re, H_Im and on the transmit         */
/* parameters).  Standard bias-corrected update; t is the 1-based step.      */
/* ------------------------------------------------------------------------ */
void or_adam(int n, double* theta, const double* g, double* m, double* v, long long t,
             double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int e = 0; e < n; ++e) {
        m[e] = b1 * m[e] + (1.0 - b1) * g[e];
        v[e] = b2 * v[e] + (1.0 - b2) * g[e] * g[e];
        double mh = m[e] / c1, vh = v[e] / c2;
        theta[e] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Transmit chain (Section III-A, READING: direct logits u, z = sigmoid(u)  */
/* mirroring the sigmoid output layer):                                     */
/*   z = 1/(1+e^-u), y = Q_A(z), x = e^{j 2 pi y}                            */
/* dL/dy = 2 pi Im(conj(x) grad_x); dL/du = dL/dy * dy/dz * z (1 - z).      */
/* ------------------------------------------------------------------------ */
void or_soft_waveform(int M, int N, const double* u, int K, const double* rho,
                      double a, double c, double* x_ri, double* dydz_out)
{
    int n = M * N;
    double* z = (double*)malloc(sizeof(double) * n);
    double* y = (double*)malloc(sizeof(double) * n);
    double* dy = (double*)malloc(sizeof(double) * n);
    for (int e = 0; e < n; ++e) z[e] = 1.0 / (1.0 + exp(-u[e]));
    or_soft_quantize(n, z, K, rho, a, c, y, dy);
    cplx* x = (cplx*)x_ri;
    for (int e = 0; e < n; ++e) x[e] = phasor(y[e]);
    if (dydz_out) for (int e = 0; e < n; ++e) dydz_out[e] = dy[e];
    free(z); free(y); free(dy);
}

void or_loss_grad_u(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                    const double* w, double eps, double snrl_db, double pnorm,
                    const double* u, int K, const double* rho, double a, double c,
                    const double* h_ri, const long long* use_cell,
                    double* terms, double* gu, double* gh_ri)
{
    int n = M * N;
    double* x = (double*)malloc(sizeof(double) * 2 * n);
    double* dy = (double*)malloc(sizeof(double) * n);
    double* gx = (double*)malloc(sizeof(double) * 2 * n);
    double* ghl = (double*)malloc(sizeof(double) * 2 * n);
    or_soft_waveform(M, N, u, K, rho, a, c, x, dy);
    or_grad_xh(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, x, h_ri, use_cell,
               terms, gx, ghl);
    const cplx* xc = (const cplx*)x;
    const cplx* gxc = (const cplx*)gx;
    for (int e = 0; e < n; ++e) {
        double gy = TWO_PI * cimag(conj(xc[e]) * gxc[e]);
        double z = 1.0 / (1.0 + exp(-u[e]));
        gu[e] = gy * dy[e] * z * (1.0 - z);
    }
    if (gh_ri) memcpy(gh_ri, ghl, sizeof(double) * 2 * n);
    free(x); free(dy); free(gx); free(ghl);
}

/* Hard waveform: x_hard(n) = e^{j 2 pi b / B}, b = q mod B. */
void or_hard_waveform(int M, int N, const double* u, int K, const double* rho, int B,
                      int* q_out, double* x_ri)
{
    int n = M * N;
    double* z = (double*)malloc(sizeof(double) * n);
    int* q = (int*)malloc(sizeof(int) * n);
    for (int e = 0; e < n; ++e) z[e] = 1.0 / (1.0 + exp(-u[e]));
    or_hard_quantize(n, z, K, rho, B, q, NULL);
    cplx* x = (cplx*)x_ri;
    for (int e = 0; e < n; ++e) x[e] = phasor((double)(q[e] % B) / (double)B);
    if (q_out) memcpy(q_out, q, sizeof(int) * n);
    free(z); free(q);
}

/* ------------------------------------------------------------------------ */
/* One outer iteration of Algorithm 1 (direct-logit transmit parameters):   */
/*   X_hard from u; N_h x {grad_H L(X_hard, H); Adam on (H_Re, H_Im);         */
/*   project (Eq. 32)}; N_x x {X_soft from u; grad_u L(X_soft, H); Adam on u} */
/* State arrays are updated in place.  losses_out receives the N_h + N_x    */
/* loss values (term[0]) in evaluation order, wpsl_out the L_WPSL values.   */
/* ------------------------------------------------------------------------ */
void or_sqngd_outer(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                    const double* w, double eps, double snrl_db, double pnorm,
                    int B, int K, const double* rho, double a, double c,
                    int n_h, int n_x, double lr_h, double lr_x,
                    double b1, double b2, double adam_eps,
                    double* u, double* h_ri,
                    double* mu, double* vu, double* mh, double* vh,
                    long long* t_x, long long* t_h,
                    double* losses_out, double* wpsl_out)
{
    int n = M * N;
    double* xh = (double*)malloc(sizeof(double) * 2 * n);
    double* gx = (double*)malloc(sizeof(double) * 2 * n);
    double* gh = (double*)malloc(sizeof(double) * 2 * n);
    double* gu = (double*)malloc(sizeof(double) * n);
    double terms[6];
    int it = 0;
    or_hard_waveform(M, N, u, K, rho, B, NULL, xh);
    for (int i = 0; i < n_h; ++i) {                       /* Step (A) */
        or_grad_xh(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, xh, h_ri, NULL,
                   terms, gx, gh);
        if (losses_out) losses_out[it] = terms[0];
        if (wpsl_out) wpsl_out[it] = terms[1];
        ++it;
        *t_h += 1;
        or_adam(2 * n, h_ri, gh, mh, vh, *t_h, lr_h, b1, b2, adam_eps);
        or_project(M, N, h_ri);
    }
    for (int j = 0; j < n_x; ++j) {                       /* Step (B) */
        or_loss_grad_u(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, u, K, rho, a, c,
                       h_ri, NULL, terms, gu, gh);
        if (losses_out) losses_out[it] = terms[0];
        if (wpsl_out) wpsl_out[it] = terms[1];
        ++it;
        *t_x += 1;
        or_adam(n, u, gu, mu, vu, *t_x, lr_x, b1, b2, adam_eps);
    }
    free(xh); free(gx); free(gh); free(gu);
}

/* ------------------------------------------------------------------------ */
/* Trainable thresholds (Section III-C allows the rho_i of Eq. 24 to be      */
/* trained; Algorithm 1 Step B updates them with Adam).                      */
/*   dQ_A/drho_i (z) = -a c (1 - tanh^2(c (z - rho_i)))                      */
/*   dL/drho_i = sum over elements e of dL/dy_e dQ_A/drho_i (z_e),           */
/* with dL/dy_e = 2 pi Im(conj(x_e) grad_x e) as in or_loss_grad_u.          */
/* grho: [K]; the other arguments as in or_loss_grad_u.                      */
/* ------------------------------------------------------------------------ */
void or_loss_grad_u_rho(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                        const double* w, double eps, double snrl_db, double pnorm,
                        const double* u, int K, const double* rho, double a, double c,
                        const double* h_ri, const long long* use_cell,
                        double* terms, double* gu, double* grho)
{
    int n = M * N;
    double* x = (double*)malloc(sizeof(double) * 2 * n);
    double* dy = (double*)malloc(sizeof(double) * n);
    double* gx = (double*)malloc(sizeof(double) * 2 * n);
    double* gh = (double*)malloc(sizeof(double) * 2 * n);
    or_soft_waveform(M, N, u, K, rho, a, c, x, dy);
    or_grad_xh(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, x, h_ri, use_cell, terms, gx, gh);
    const cplx* xc = (const cplx*)x;
    const cplx* gxc = (const cplx*)gx;
    for (int i = 0; i < K; ++i) grho[i] = 0.0;
    for (int e = 0; e < n; ++e) {
        double gy = TWO_PI * cimag(conj(xc[e]) * gxc[e]);
        double z = 1.0 / (1.0 + exp(-u[e]));
        if (gu) gu[e] = gy * dy[e] * z * (1.0 - z);
        for (int i = 0; i < K; ++i) {
            double t = tanh(c * (z - rho[i]));
            grho[i] += gy * (-a * c * (1.0 - t * t));
        }
    }
    free(x); free(dy); free(gx); free(gh);
}

/* Euclidean projection onto the ordered thresholds inside [0, 1]
 * (Section III-C requires them ordered; READING: the nearest set
 * 0 <= rho_0 <= ... <= rho_{K-1} <= 1): isotonic regression by pooling
 * adjacent violators (Barlow et al. 1972), then clipping to [0, 1] (the
 * clipped isotonic fit is the projection onto the intersection).  In place. */
void or_project_thresholds(int K, double* rho)
{
    double* val = (double*)malloc(sizeof(double) * K);
    int* cnt = (int*)malloc(sizeof(int) * K);
    int nb = 0;
    for (int i = 0; i < K; ++i) {
        val[nb] = rho[i];
        cnt[nb] = 1;
        ++nb;
        while (nb > 1 && val[nb - 2] > val[nb - 1]) {   /* pool the violating pair of blocks */
            double tot = val[nb - 2] * cnt[nb - 2] + val[nb - 1] * cnt[nb - 1];
            cnt[nb - 2] += cnt[nb - 1];
            val[nb - 2] = tot / cnt[nb - 2];
            --nb;
        }
    }
    int i = 0;
    for (int b = 0; b < nb; ++b) {
        double v = val[b] < 0.0 ? 0.0 : (val[b] > 1.0 ? 1.0 : val[b]);
        for (int r = 0; r < cnt[b]; ++r) rho[i++] = v;
    }
    free(val); free(cnt);
}

/* One outer iteration of Algorithm 1 with trainable thresholds: as
 * or_sqngd_outer, and every Step-B evaluation also takes dL/drho, applies
 * Adam to rho (same step counter as u, learning rate lr_rho, moments mr, vr)
 * and projects rho (or_project_thresholds).  rho is updated in place. */
void or_sqngd_outer_rho(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                        const double* w, double eps, double snrl_db, double pnorm,
                        int B, int K, double* rho, double a, double c,
                        int n_h, int n_x, double lr_h, double lr_x, double lr_rho,
                        double b1, double b2, double adam_eps,
                        double* u, double* h_ri,
                        double* mu, double* vu, double* mh, double* vh, double* mr, double* vr,
                        long long* t_x, long long* t_h,
                        double* losses_out, double* wpsl_out)
{
    int n = M * N;
    double* xh = (double*)malloc(sizeof(double) * 2 * n);
    double* gx = (double*)malloc(sizeof(double) * 2 * n);
    double* gh = (double*)malloc(sizeof(double) * 2 * n);
    double* gu = (double*)malloc(sizeof(double) * n);
    double* gr = (double*)malloc(sizeof(double) * K);
    double terms[6];
    int it = 0;
    or_hard_waveform(M, N, u, K, rho, B, NULL, xh);
    for (int i = 0; i < n_h; ++i) {                       /* Step (A) */
        or_grad_xh(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, xh, h_ri, NULL,
                   terms, gx, gh);
        if (losses_out) losses_out[it] = terms[0];
        if (wpsl_out) wpsl_out[it] = terms[1];
        ++it;
        *t_h += 1;
        or_adam(2 * n, h_ri, gh, mh, vh, *t_h, lr_h, b1, b2, adam_eps);
        or_project(M, N, h_ri);
    }
    for (int j = 0; j < n_x; ++j) {                       /* Step (B): u and rho */
        or_loss_grad_u_rho(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, u, K, rho, a, c,
                           h_ri, NULL, terms, gu, gr);
        if (losses_out) losses_out[it] = terms[0];
        if (wpsl_out) wpsl_out[it] = terms[1];
        ++it;
        *t_x += 1;
        or_adam(n, u, gu, mu, vu, *t_x, lr_x, b1, b2, adam_eps);
        or_adam(K, rho, gr, mr, vr, *t_x, lr_rho, b1, b2, adam_eps);
        or_project_thresholds(K, rho);
    }
    free(xh); free(gx); free(gh); free(gu); free(gr);
}

/* ------------------------------------------------------------------------ */
/* SQNAF (Section IV): the delay-Doppler WPSL objective with no receive-     */
/* filter optimisation -- every filter is the waveform itself, h = x, so     */
/* the loss is L(x, x) and, by the chain rule through both arguments,        */
/*   grad L(x, x) = grad_x L(x, h) + grad_h L(x, h)   at h = x.              */
/* Same real-pair convention and use_cell meaning as or_grad_xh.             */
/* ------------------------------------------------------------------------ */
void or_grad_matched(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                     const double* w, double eps, double snrl_db, double pnorm,
                     const double* x_ri, const long long* use_cell,
                     double* terms, double* g_ri)
{
    int n = M * N;
    double* gh = (double*)malloc(sizeof(double) * 2 * n);
    or_grad_xh(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, x_ri, x_ri, use_cell,
               terms, g_ri, gh);
    for (int e = 0; e < 2 * n; ++e) g_ri[e] += gh[e];
    free(gh);
}

/* The transmit chain of Section III-A on the SQNAF loss: x = soft(u), the
 * gradient of L(x, x) mapped to the logits as in or_loss_grad_u. */
void or_loss_grad_u_matched(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                            const double* w, double eps, double snrl_db, double pnorm,
                            const double* u, int K, const double* rho, double a, double c,
                            const long long* use_cell, double* terms, double* gu)
{
    int n = M * N;
    double* x = (double*)malloc(sizeof(double) * 2 * n);
    double* dy = (double*)malloc(sizeof(double) * n);
    double* g = (double*)malloc(sizeof(double) * 2 * n);
    or_soft_waveform(M, N, u, K, rho, a, c, x, dy);
    or_grad_matched(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, x, use_cell, terms, g);
    const cplx* xc = (const cplx*)x;
    const cplx* gc = (const cplx*)g;
    for (int e = 0; e < n; ++e) {
        double gy = TWO_PI * cimag(conj(xc[e]) * gc[e]);
        double z = 1.0 / (1.0 + exp(-u[e]));
        gu[e] = gy * dy[e] * z * (1.0 - z);
    }
    free(x); free(dy); free(g);
}

/* One outer iteration of SQNAF: Step (A) of Algorithm 1 is skipped (there
 * is no filter to update); the hard design is scored once, L(X_hard,
 * X_hard), then N_x x {X_soft from u; grad_u L(X_soft, X_soft); Adam on u}.
 * losses_out / wpsl_out receive 1 + N_x values: the score first. */
void or_sqnaf_outer(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                    const double* w, double eps, double snrl_db, double pnorm,
                    int B, int K, const double* rho, double a, double c,
                    int n_x, double lr_x, double b1, double b2, double adam_eps,
                    double* u, double* mu, double* vu, long long* t_x,
                    double* losses_out, double* wpsl_out)
{
    int n = M * N;
    double* xh = (double*)malloc(sizeof(double) * 2 * n);
    double* gu = (double*)malloc(sizeof(double) * n);
    double* pm = (double*)malloc(sizeof(double) * M);
    double terms[6];
    long long cells[2];
    or_hard_waveform(M, N, u, K, rho, B, NULL, xh);
    or_loss(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, xh, xh, terms, pm, cells);
    if (losses_out) losses_out[0] = terms[0];
    if (wpsl_out) wpsl_out[0] = terms[1];
    for (int j = 0; j < n_x; ++j) {
        or_loss_grad_u_matched(M, N, L, nu, k_lo, k_hi, w, eps, snrl_db, pnorm, u, K, rho, a, c,
                               NULL, terms, gu);
        if (losses_out) losses_out[1 + j] = terms[0];
        if (wpsl_out) wpsl_out[1 + j] = terms[1];
        *t_x += 1;
        or_adam(n, u, gu, mu, vu, *t_x, lr_x, b1, b2, adam_eps);
    }
    free(xh); free(gu); free(pm);
}

/* ------------------------------------------------------------------------ */
/* Acceptance metrics: PSLR (Eq. 48) of the auto and cross terms over the    */
/* ROI (cells of positive weight; auto excludes tau = 0 as in Eq. 8) and the */
/* SNRL of Eq. 10 for every m.                                               */
/* out[0] = APSL dB, out[1] = CPSL dB, out[2] = PSLR dB (max of the two),     */
/* out[3] = max_m SNRL dB; snrl[m] per waveform (may be NULL).               */
/* ------------------------------------------------------------------------ */
void or_metrics(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                const double* w, const double* x_ri, const double* h_ri,
                double* out, double* snrl)
{
    or_cfg c = { M, N, L, k_lo, k_hi, nu, NULL, 0.0, 0.0, 0.0 };
    const cplx* x = (const cplx*)x_ri;
    const cplx* h = (const cplx*)h_ri;
    int D = k_hi - k_lo + 1;
    double psl[2] = { 0, 0 };
    long long rows = (long long)M * M * D;
    cplx* E = phasor_table(N, L, nu);
    double* rowmax = (double*)calloc((size_t)rows, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
    for (long long r = 0; r < rows; ++r) {
        int d = (int)(r % D), pair = (int)(r / D), m = pair / M, l = pair % M;
        int k = k_lo + d;
        if (cell_class(m, l, k) < 0) continue;
        for (int j = 0; j < L; ++j) {
            if (w && !(w[(size_t)d * L + j] > 0)) continue;
            double v = cabs(af_cell_tab(N, x + (size_t)m * N, h + (size_t)l * N, k, E + (size_t)j * N));
            if (v > rowmax[r]) rowmax[r] = v;
        }
    }
    for (long long r = 0; r < rows; ++r) {
        int d = (int)(r % D), pair = (int)(r / D), m = pair / M, l = pair % M;
        int cls = cell_class(m, l, k_lo + d);
        if (cls >= 0 && rowmax[r] > psl[cls]) psl[cls] = rowmax[r];
    }
    free(rowmax); free(E);
    out[0] = 20.0 * log10(psl[0] / (double)N);
    out[1] = 20.0 * log10(psl[1] / (double)N);
    out[2] = out[0] > out[1] ? out[0] : out[1];
    double smax = -1e300;
    for (int m = 0; m < M; ++m) {
        double ex = 0, eh = 0;
        cplx ip = 0;
        for (int n = 0; n < N; ++n) {
            cplx xv = x[(size_t)m * N + n], hv = h[(size_t)m * N + n];
            ex += creal(xv * conj(xv)); eh += creal(hv * conj(hv));
            ip += conj(xv) * hv;                                        /* x^H h */
        }
        double s = 10.0 * log10(ex * eh / (creal(ip * conj(ip))));     /* Eq. 10 */
        if (snrl) snrl[m] = s;
        if (s > smax) smax = s;
    }
    out[3] = smax;
    (void)c;
}

/* ------------------------------------------------------------------------ */
/* Gradient of Eq. 42 when the exact max is taken at a known cell, without   */
/* scanning the grid (for grids too large to scan): the sidelobe term at     */
/* that cell (weight w_cell) plus the SNRL term.  Same convention as         */
/* or_grad_xh; chi_out receives chi at the cell.                             */
/* ------------------------------------------------------------------------ */
void or_grad_at_cell(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                     double w_cell, double eps, double snrl_db,
                     const double* x_ri, const double* h_ri, long long cell,
                     double* chi_out, double* gx_ri, double* gh_ri)
{
    or_cfg c = { M, N, L, k_lo, k_hi, nu, NULL, eps, snrl_db, 0.0 };
    const cplx* x = (const cplx*)x_ri;
    const cplx* h = (const cplx*)h_ri;
    cplx* gx = (cplx*)gx_ri;
    cplx* gh = (cplx*)gh_ri;
    int D = k_hi - k_lo + 1;
    memset(gx, 0, sizeof(cplx) * (size_t)M * N);
    memset(gh, 0, sizeof(cplx) * (size_t)M * N);
    int j = (int)(cell % L), d = (int)((cell / L) % D);
    int pair = (int)(cell / ((long long)L * D));
    cplx a = af_cell(N, x + (size_t)(pair / M) * N, h + (size_t)(pair % M) * N, k_lo + d, nu[j]);
    if (chi_out) { chi_out[0] = creal(a); chi_out[1] = cimag(a); }
    double mag = cabs(a);
    if (mag > 0) add_cell_grad(&c, x, h, cell, eps * w_cell * a / mag, gx, gh);
    double ptar = pow(10.0, -snrl_db / 20.0);
    for (int m = 0; m < M; ++m) {
        cplx a00 = 0;
        for (int n = 0; n < N; ++n) a00 += x[(size_t)m * N + n] * conj(h[(size_t)m * N + n]);
        double am = cabs(a00);
        if (am <= 0) continue;
        cplx G = (1.0 - eps) * (2.0 / M) * (am / N - ptar) / (double)N * a00 / am;
        for (int n = 0; n < N; ++n) {
            gx[(size_t)m * N + n] += G * h[(size_t)m * N + n];
            gh[(size_t)m * N + n] += conj(G) * x[(size_t)m * N + n];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Losses at perturbed inputs, for central finite differences at full size. */
/* Coordinate c replaces one sample -- x_row(col) when target[c] = 0,        */
/* h_row(col) when target[c] = 1 -- by vp[c] (the + side) and by vm[c] (the  */
/* - side).  Eq. 6 is linear in x_m(n) and in conj(h_l(p)), so              */
/*   x_m(n) -> x_m(n) + delta  moves chi_ml(k, nu) by                        */
/*                delta conj(h_l(n+k)) e^{j 2 pi nu n}         (all l, k, nu) */
/*   h_l(p) -> h_l(p) + delta  moves chi_ml(k, nu) by                        */
/*                x_m(p-k) conj(delta) e^{j 2 pi nu (p-k)}     (all m, k, nu) */
/* a rank-one change that touches only the M pairs of one row (or column)   */
/* of the pair grid.  Every other pair keeps the class peak (and p-norm sum) */
/* of the unperturbed grid, so each perturbed loss costs one pass over M     */
/* pairs' cells instead of a full evaluation.  The SNRL term (Eqs. 38, 41)   */
/* is recomputed from the perturbed inputs, and the loss assembled as in     */
/* or_loss (Eqs. 7-9, 37, 42).  The test suite checks this routine against   */
/* or_loss on explicitly perturbed inputs.                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    double vmax;   /* max of w|chi| over the pair's cells of its class */
    double psum;   /* sum of (w|chi| / vmax)^p over them (p-norm only) */
    int any;
} fd_stat;

/* Fold (v, s) into a running (vmax, psum): both sums rescaled to the larger max. */
static void fd_fold(double pnorm, fd_stat* a, double v, double s)
{
    if (!a->any) { a->vmax = v; a->psum = s; a->any = 1; return; }
    if (pnorm <= 0) { if (v > a->vmax) a->vmax = v; return; }
    if (v > a->vmax) {
        a->psum = (a->vmax > 0 ? a->psum * pow(a->vmax / v, pnorm) : 0.0) + s;
        a->vmax = v;
    } else {
        a->psum += (v > 0 ? s * pow(v / a->vmax, pnorm) : 0.0);
    }
}

/* Statistics of one pair (m, l) whose grid is chi[D][L] plus the rank-one
 * term dk[d] * ej[j] (dk = NULL: unperturbed).  Rows are reduced in order. */
static fd_stat fd_pair_stat(const or_cfg* c, int m, int l, const cplx* chi, const cplx* dk, const cplx* ej,
                            double* rmax, double* rsum)
{
    int L = c->L, D = c->k_hi - c->k_lo + 1;
#pragma omp parallel for schedule(static)
    for (int d = 0; d < D; ++d) {
        rmax[d] = -1.0; rsum[d] = 0.0;
        if (cell_class(m, l, c->k_lo + d) < 0) continue;
        const cplx* row = chi + (size_t)d * L;
        double vm = -1.0;
        for (int j = 0; j < L; ++j) {
            double w = cell_weight(c, d, j);
            if (w <= 0) continue;
            cplx a = dk ? row[j] + dk[d] * ej[j] : row[j];
            double v = w * cabs(a);
            if (v > vm) vm = v;
        }
        rmax[d] = vm;
        if (c->pnorm > 0 && vm > 0) {
            double s = 0;
            for (int j = 0; j < L; ++j) {
                double w = cell_weight(c, d, j);
                if (w <= 0) continue;
                cplx a = dk ? row[j] + dk[d] * ej[j] : row[j];
                s += pow(w * cabs(a) / vm, c->pnorm);
            }
            rsum[d] = s;
        }
    }
    fd_stat st = { 0.0, 0.0, 0 };
    for (int d = 0; d < D; ++d)
        if (rmax[d] >= 0) fd_fold(c->pnorm, &st, rmax[d], rsum[d]);
    return st;
}

void or_fd_losses(int M, int N, int L, const double* nu, int k_lo, int k_hi,
                  const double* w, double eps, double snrl_db, double pnorm,
                  const double* x_ri, const double* h_ri, int ncoord,
                  const int* target, const int* row, const int* col,
                  const double* vp_ri, const double* vm_ri,
                  double* loss_p, double* loss_m)
{
    or_cfg c = { M, N, L, k_lo, k_hi, nu, w, eps, snrl_db, pnorm };
    const cplx* x = (const cplx*)x_ri;
    const cplx* h = (const cplx*)h_ri;
    const cplx* vp = (const cplx*)vp_ri;
    const cplx* vmn = (const cplx*)vm_ri;
    int D = k_hi - k_lo + 1, P = M * M;
    cplx* E = phasor_table(N, L, nu);
    cplx* chi = (cplx*)malloc(sizeof(cplx) * (size_t)D * L);
    cplx* dk = (cplx*)malloc(sizeof(cplx) * (size_t)D);
    cplx* ej = (cplx*)malloc(sizeof(cplx) * (size_t)L);
    double* rmax = (double*)malloc(sizeof(double) * D);
    double* rsum = (double*)malloc(sizeof(double) * D);
    fd_stat* base = (fd_stat*)calloc((size_t)P, sizeof(fd_stat));
    fd_stat* pert = (fd_stat*)calloc((size_t)ncoord * 2 * P, sizeof(fd_stat));

    for (int pair = 0; pair < P; ++pair) {
        int m = pair / M, l = pair % M;
        /* Eq. 6 on every cell of this pair */
#pragma omp parallel for schedule(static)
        for (int d = 0; d < D; ++d)
            for (int j = 0; j < L; ++j)
                chi[(size_t)d * L + j] = af_cell_tab(N, x + (size_t)m * N, h + (size_t)l * N, k_lo + d,
                                                     E + (size_t)j * N);
        base[pair] = fd_pair_stat(&c, m, l, chi, NULL, NULL, rmax, rsum);
        for (int ci = 0; ci < ncoord; ++ci) {
            int r = row[ci], n0 = col[ci];
            int touches = (target[ci] == 0) ? (r == m) : (r == l);
            if (!touches) continue;
            for (int side = 0; side < 2; ++side) {
                cplx v = side == 0 ? vp[ci] : vmn[ci];
                if (target[ci] == 0) {
                    cplx delta = v - x[(size_t)m * N + n0];
                    for (int d = 0; d < D; ++d) {
                        int q = n0 + k_lo + d;
                        dk[d] = (q >= 0 && q < N) ? delta * conj(h[(size_t)l * N + q]) : 0.0;
                    }
                    for (int j = 0; j < L; ++j) ej[j] = E[(size_t)j * N + n0];
                } else {
                    /* h_l(p0) changes: the sample n = p0 - k of row k, phasor e^{j 2 pi nu n} */
                    cplx delta = v - h[(size_t)l * N + n0];
                    for (int d = 0; d < D; ++d) dk[d] = 0.0;
                    /* the phasor depends on n = p0 - k, so the term is not a product of a
                     * row factor and a column factor: handle it row by row */
                    fd_stat st = { 0.0, 0.0, 0 };
#pragma omp parallel for schedule(static)
                    for (int d = 0; d < D; ++d) {
                        int k = k_lo + d, n = n0 - k;
                        rmax[d] = -1.0; rsum[d] = 0.0;
                        if (cell_class(m, l, k) < 0) continue;
                        cplx a0 = (n >= 0 && n < N) ? x[(size_t)m * N + n] * conj(delta) : 0.0;
                        const cplx* row_ = chi + (size_t)d * L;
                        double vmx = -1.0;
                        for (int j = 0; j < L; ++j) {
                            double wt = cell_weight(&c, d, j);
                            if (wt <= 0) continue;
                            cplx a = (n >= 0 && n < N) ? row_[j] + a0 * E[(size_t)j * N + n] : row_[j];
                            double vv = wt * cabs(a);
                            if (vv > vmx) vmx = vv;
                        }
                        rmax[d] = vmx;
                        if (pnorm > 0 && vmx > 0) {
                            double s = 0;
                            for (int j = 0; j < L; ++j) {
                                double wt = cell_weight(&c, d, j);
                                if (wt <= 0) continue;
                                cplx a = (n >= 0 && n < N) ? row_[j] + a0 * E[(size_t)j * N + n] : row_[j];
                                s += pow(wt * cabs(a) / vmx, pnorm);
                            }
                            rsum[d] = s;
                        }
                    }
                    for (int d = 0; d < D; ++d)
                        if (rmax[d] >= 0) fd_fold(pnorm, &st, rmax[d], rsum[d]);
                    pert[((size_t)ci * 2 + side) * P + pair] = st;
                    continue;
                }
                pert[((size_t)ci * 2 + side) * P + pair] = fd_pair_stat(&c, m, l, chi, dk, ej, rmax, rsum);
            }
        }
    }

    double ptar = pow(10.0, -snrl_db / 20.0);                       /* Eq. 39 */
    for (int ci = 0; ci < ncoord; ++ci) {
        for (int side = 0; side < 2; ++side) {
            fd_stat cls[2] = { { 0.0, 0.0, 0 }, { 0.0, 0.0, 0 } };
            for (int pair = 0; pair < P; ++pair) {
                int m = pair / M, l = pair % M;
                int touched = (target[ci] == 0) ? (row[ci] == m) : (row[ci] == l);
                const fd_stat* s = touched ? &pert[((size_t)ci * 2 + side) * P + pair] : &base[pair];
                if (s->any) fd_fold(pnorm, &cls[m == l ? 0 : 1], s->vmax, s->psum);
            }
            double v[2];
            for (int k = 0; k < 2; ++k) {                             /* Eqs. 8-9 (or their p-norms) */
                if (!cls[k].any) v[k] = 0.0;
                else if (pnorm > 0) v[k] = cls[k].vmax * pow(cls[k].psum, 1.0 / pnorm);
                else v[k] = cls[k].vmax;
            }
            double lw = v[0] >= v[1] ? v[0] : v[1];                   /* Eq. 37 */
            cplx nv = side == 0 ? vp[ci] : vmn[ci];
            double ls = 0;
            for (int m = 0; m < M; ++m) {
                cplx a00 = 0;
                for (int n = 0; n < N; ++n) {
                    cplx xv = x[(size_t)m * N + n], hv = h[(size_t)m * N + n];
                    if (m == row[ci] && n == col[ci]) {
                        if (target[ci] == 0) xv = nv; else hv = nv;
                    }
                    a00 += conj(hv) * xv;
                }
                double dev = cabs(a00) / (double)N - ptar;            /* Eq. 38 */
                ls += dev * dev;
            }
            ls /= (double)M;                                          /* Eq. 41 */
            double loss = eps * lw + (1.0 - eps) * ls;                /* Eq. 42 */
            if (side == 0) loss_p[ci] = loss; else loss_m[ci] = loss;
        }
    }
    free(E); free(chi); free(dk); free(ej); free(rmax); free(rsum); free(base); free(pert);
}
