"""Split-BF16 tensor-core path (AF_PATH_SPLIT_BF16) vs the FP64 oracle.

Tolerances for this path: |chi| error <= 1e-4 of the mainlobe (max |chi|),
PSL (each class) within 0.1 dB, the winning cell a maximum of the oracle's
grid within that bound, and the gradient at the winning cell within 1e-4 of
its scale.  Inputs are rounded to complex64 before either side sees them.
"""
import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CHI_TOL = 1e-4        # of the mainlobe
DB_TOL = 0.1


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import api as a
    return a


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pair(orc, seed, M, N, noise=0.3):
    x = wl.unit_phasors(seed, M, N).astype(np.complex64)
    h = orc.project(x.astype(np.complex128) + noise * wl.complex_normal(seed, M, N)).astype(np.complex64)
    return x, h


def _ctx(api, M, N, B, nu, k_lo, k_hi, **kw):
    kw.setdefault("r_n", 100)
    c = api.Context(M, N, B, nu, k_lo, k_hi, path=api.AF_PATH_SPLIT_BF16, **kw)
    assert c.path == api.AF_PATH_SPLIT_BF16
    return c


SPLIT_CASES = [
    # M, N, nu, k_lo, k_hi
    (2, 100, wl.window_grid(0.05, 64), -40, 40),              # one delay tile, 64 bins
    (3, 300, wl.window_grid(0.1, 40), -299, 299),             # 5 delay tiles, ragged rows and bins
    (1, 77, wl.window_grid(0.2, 16), -76, 76),                # N not a multiple of the 32-sample chunk
    (2, 64, wl.window_grid(0.02, 100), -63, 63),              # 128-bin column tile, 28 padded bins
    (1, 50, np.sort(wl.uniform(5, 200, 1) - 0.5), -30, 49),   # two column tiles, irregular grid
    (2, 130, np.array([0.0]), -129, 129),                     # zero-Doppler row (L = 1)
    (1, 2, np.array([-0.1, 0.25]), -1, 1),                    # smallest N
]


@pytest.mark.parametrize("case", SPLIT_CASES)
def test_split_ambiguity_matches_oracle(api, orc, case):
    M, N, nu, k_lo, k_hi = case
    x, h = _pair(orc, 500 + N, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi)
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    err = np.max(np.abs(chi - ref))
    assert err <= CHI_TOL * np.max(np.abs(ref)), err / np.max(np.abs(ref))
    ctx.af_sync()


def _check_terms(orc, ctx, x, h, nu, k_lo, k_hi, eps, snrl_db, weights=None):
    M, N = x.shape
    gx = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h), grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    r = orc.loss(x, h, nu, k_lo, k_hi, weights=weights, eps=eps, snrl_db=snrl_db)
    # the mainlobe in the loss's units: max w |chi| over the weighted grid is
    # bounded by max(w) N for unimodular x and energy-N filters
    wmax = (1.0 / N) if weights is None else float(np.max(weights))
    tol = CHI_TOL * wmax * N
    for gi, key in ((2, "wapsl"), (3, "wcpsl")):
        assert abs(t[gi] - r[key]) <= tol, (key, t[gi], r[key])
        if r[key] > 0:
            assert abs(20 * np.log10(t[gi] / r[key])) <= DB_TOL
    np.testing.assert_allclose(t[8:8 + M], r["p"], atol=1e-6)      # chi_mm(0,0) is FP64 on every path
    assert abs(t[0] - r["loss"]) <= tol
    cls = int(t[5])
    cell = int(t[6 + cls])
    assert cell >= 0
    full = orc.ambiguity(x, h, nu, k_lo, k_hi).reshape(-1)
    D, L = k_hi - k_lo + 1, nu.size
    d, j = (cell // L) % D, cell % L
    w = (1.0 / N) if weights is None else weights[d, j]
    assert w * abs(full[cell]) >= r["wpsl"] - tol
    _, ogx, ogh = orc.grad_xh(x, h, nu, k_lo, k_hi, weights=weights, eps=eps, snrl_db=snrl_db, use_cell=cell)
    scale = max(np.max(np.abs(ogx)), np.max(np.abs(ogh)))
    assert np.max(np.abs(gx.cpu().numpy() - ogx)) <= 1e-4 * scale
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 1e-4 * scale
    return t, r


@pytest.mark.parametrize("case", SPLIT_CASES[:5])
def test_split_loss_and_gradient(api, orc, case):
    M, N, nu, k_lo, k_hi = case
    x, h = _pair(orc, 600 + N, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi, eps=0.2, snrl_db=1.0)
    _check_terms(orc, ctx, x, h, nu, k_lo, k_hi, 0.2, 1.0)


def test_split_weight_map(api, orc):
    M, N = 2, 96
    nu = wl.window_grid(0.08, 48)
    k_lo, k_hi = -95, 95
    D, L = k_hi - k_lo + 1, nu.size
    wts = (wl.uniform(19, D * L, 3).reshape(D, L) / N).astype(np.float32).astype(np.float64)
    wts[:, :6] = 0.0
    x, h = _pair(orc, 19, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi, weights=wts, eps=0.5)
    _check_terms(orc, ctx, x, h, nu, k_lo, k_hi, 0.5, 0.5, weights=wts)


def test_split_agrees_with_fp32_dft_path(api, orc):
    """Same inputs through the SIMT FP32 DFT and the tensor-core path."""
    M, N = 2, 256
    nu = wl.window_grid(0.05, 64)
    x, h = _pair(orc, 23, M, N)
    c_split = _ctx(api, M, N, 4, nu, -200, 200)
    c_dft = api.Context(M, N, 4, nu, -200, 200, r_n=100, path=api.AF_PATH_DFT)
    a = c_split.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    b = c_dft.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    assert np.max(np.abs(a - b)) <= CHI_TOL * N


def test_split_optimiser_step_runs(api, orc):
    """Outer iterations of Algorithm 1 on the tensor-core path: the first
    evaluation (identical inputs) logs the FP32 DFT path's loss within the
    split tolerance, and the run stays finite and keeps a best design."""
    M, N, B, r_n = 2, 128, 8, 100
    nu = wl.window_grid(0.05, 32)
    b = wl.phase_indices(29, M, N, B)
    u0 = orc.init_logits(b, B, r_n).astype(np.float32)
    h0 = orc.project(np.exp(2j * np.pi * b / B)).astype(np.complex64)
    logs = []
    for path in (api.AF_PATH_SPLIT_BF16, api.AF_PATH_DFT):
        ctx = api.Context(M, N, B, nu, -60, 60, r_n=r_n, path=path, n_h=3, n_x=3)
        st = api.SqngdState.create(_dev(u0), _dev(h0))
        log = ctx.sqngd_step(st, 5)
        ctx.af_sync()
        assert np.all(np.isfinite(log))
        assert np.all(np.isfinite(st.u.cpu().numpy())) and np.all(np.isfinite(st.h.cpu().numpy()))
        assert st.best.cpu().numpy()[0] < np.inf
        logs.append(log)
    assert abs(logs[0][0, 0, 0] - logs[1][0, 0, 0]) <= CHI_TOL


def _sampled_cells(seed, total, n=3000):
    return np.unique((wl.uniform(seed, n, 4) * total).astype(np.int64))


def test_split_full_size_precision(api, orc):
    """M=8, N=1024, |k| <= 255, 64 bins on |nu| <= 0.05 -- the launch the
    benchmark times on this path: sampled cells, both PSL classes, the
    winning cell and the gradient there, all against the oracle."""
    w = wl.precision()
    x, h = _pair(orc, 41, w.M, w.N)
    ctx = _ctx(api, w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db)
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).reshape(-1)
    cells = _sampled_cells(41, chi.numel())
    got = chi[torch.from_numpy(cells).cuda()].cpu().numpy()
    ref = orc.ambiguity_cells(x, h, w.nu, w.k_lo, w.k_hi, cells)
    assert np.max(np.abs(got - ref)) <= CHI_TOL * w.N
    _check_terms(orc, ctx, x, h, w.nu, w.k_lo, w.k_hi, w.eps, w.snrl_db)


@pytest.mark.parametrize("shape", [("16x4x2", "1"), ("32x2x2", "2"), ("16x4x2", "2"),
                                   ("32x4x2", "2"), ("16x8x4", "2")])
def test_split_pipeline_variants(api, orc, shape, monkeypatch):
    """Other pipeline shapes of the tensor-core kernel (samples per stage x
    B stages x A stages, pairs per CTA) give the same chi and loss."""
    cfg, tiles = shape
    monkeypatch.setenv("SQNGD_GEMM_CFG", cfg)
    monkeypatch.setenv("SQNGD_GEMM_TILES", tiles)
    M, N, nu, k_lo, k_hi = 4, 300, wl.window_grid(0.1, 40), -299, 299
    x, h = _pair(orc, 700 + N, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi, eps=0.2, snrl_db=1.0)
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    assert np.max(np.abs(chi - ref)) <= CHI_TOL * np.max(np.abs(ref))
    _check_terms(orc, ctx, x, h, nu, k_lo, k_hi, 0.2, 1.0)


@pytest.mark.parametrize("lb", ["16", "32", "64", "128"])
def test_split_column_tile_widths(api, orc, lb, monkeypatch):
    """Every column-tile width (16 to 128 bins per tile; the library narrows
    the tiles when too few exist to fill the GPU) gives the oracle's chi,
    terms, cell and gradient on a 128-bin window with a ragged delay tile."""
    monkeypatch.setenv("SQNGD_GEMM_LB", lb)
    M, N, nu, k_lo, k_hi = 2, 330, wl.window_grid(0.1, 128), -150, 150
    x, h = _pair(orc, 800 + int(lb), M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi, eps=0.2, snrl_db=1.0)
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    assert np.max(np.abs(chi - ref)) <= CHI_TOL * np.max(np.abs(ref))
    _check_terms(orc, ctx, x, h, nu, k_lo, k_hi, 0.2, 1.0)


def test_pipeline_wait_timeout_is_reported_and_device_stays_usable(api, orc, monkeypatch):
    """Failure detection without a fault: with the test hook the MMA issuer
    waits on a barrier that nothing completes; the bounded wait (50 ms) gives
    up, the CTA drains and exits, af_sync reports AF_ERR_TIMEOUT, and the
    next context on the same device computes correct results."""
    M, N, nu, k_lo, k_hi = 1, 64, wl.window_grid(0.1, 16), -10, 10
    x, h = _pair(orc, 900, M, N)
    monkeypatch.setenv("SQNGD_GEMM_TEST_STALL", "1")
    bad = _ctx(api, M, N, 4, nu, k_lo, k_hi)
    bad.af_forward(_dev(x), _dev(h))
    with pytest.raises(api.AfError, match="AF_ERR_TIMEOUT"):
        bad.af_sync()
    bad.af_sync()                    # the flag is cleared once reported
    bad.close()
    monkeypatch.delenv("SQNGD_GEMM_TEST_STALL")
    good = _ctx(api, M, N, 4, nu, k_lo, k_hi)
    chi = good.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    assert np.max(np.abs(chi - ref)) <= CHI_TOL * np.max(np.abs(ref))
    good.af_sync()


def _split_work(M, N, nu, k_lo, k_hi, spc=32):
    """Sample chunks of all tiles (the split schedule's work) with the widest
    column tile, and the tiles' count: as the library plans them."""
    L = len(nu)
    lb = 16
    while lb < L and lb < 128:
        lb *= 2
    n_ct = (L + lb - 1) // lb
    D = k_hi - k_lo + 1
    total = 0
    for b in range((D + 127) // 128):
        k_first, k_last = k_lo + 128 * b, k_lo + min(D, 128 * b + 128) - 1
        n_begin, n_end = max(0, -k_last), min(N, N - k_first)
        total += (n_end + spc - 1) // spc - n_begin // spc
    return M * M * n_ct * total


@pytest.mark.parametrize("case,ctas", [
    ((2, 100, wl.window_grid(0.05, 64), -40, 40), "3"),     # tiles of 4 chunks in 2-3 pieces
    ((2, 100, wl.window_grid(0.05, 64), -40, 40), "16"),    # one chunk per CTA: 4 pieces per tile
    ((3, 300, wl.window_grid(0.1, 40), -299, 299), "11"),   # several whole and split tiles per CTA
    ((3, 300, wl.window_grid(0.1, 40), -299, 299), "97"),
    ((1, 50, np.sort(wl.uniform(5, 200, 1) - 0.5), -30, 49), "3"),   # two column tiles
])
def test_split_schedule_matches_oracle(api, orc, case, ctas, monkeypatch):
    """The split schedule forced onto small problems (the library enables it by
    itself when more tiles than SMs do not fill whole waves): CTAs share the
    chunk work, split tiles are finished by their last piece.  chi on every
    cell, the loss terms, the winning cell and the gradient match the oracle,
    and a second evaluation gives bit-identical results (the pieces are added
    in a fixed order whichever CTA finishes the tile)."""
    M, N, nu, k_lo, k_hi = case
    assert _split_work(M, N, nu, k_lo, k_hi) >= int(ctas)   # every CTA gets work: the schedule is used
    monkeypatch.setenv("SQNGD_GEMM_SPLIT_CTAS", ctas)
    x, h = _pair(orc, 1000 + N + int(ctas), M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi, eps=0.2, snrl_db=1.0)
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    assert np.max(np.abs(chi - ref)) <= CHI_TOL * np.max(np.abs(ref))
    _check_terms(orc, ctx, x, h, nu, k_lo, k_hi, 0.2, 1.0)
    outs = []
    for _ in range(2):
        gx = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        gh = torch.empty_like(gx)
        terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h), grad_x=gx, grad_h=gh)
        ctx.af_sync()
        outs.append((terms.cpu().numpy(), gx.cpu().numpy(), gh.cpu().numpy()))
    for u, v in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(u, v)
    ctx.close()


def test_split_schedule_on_and_off_agree(api, orc, monkeypatch):
    """The learned workload (64 tiles: the split schedule is the default there)
    with and without the schedule: the same PSL classes and winning class."""
    w = wl.learned()
    x, h = _pair(orc, 1234, w.M, w.N)
    res = []
    for flag in ("1", "0"):
        monkeypatch.setenv("SQNGD_GEMM_SPLIT", flag)
        ctx = _ctx(api, w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi)
        terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h))
        ctx.af_sync()
        res.append(terms.cpu().numpy())
        ctx.close()
    a, b = res
    np.testing.assert_allclose(a[[1, 2, 3]], b[[1, 2, 3]], rtol=1e-5)
    assert int(a[5]) == int(b[5])
