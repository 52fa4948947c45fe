"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP32 path): |chi| error <= 1e-5 of the mainlobe N; PSL difference
<= 0.05 dB; quantizer indices bit-exact given the same FP32 continuous phases.
Inputs are rounded to complex64 before they reach either side, so both see
identical values.
"""
import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CHI_TOL = 1e-5        # of the mainlobe N
DB_TOL = 0.05


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import api as a
    return a


def _c64(a):
    return np.asarray(a).astype(np.complex64)


def _dev(a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a).cuda()


def _pair(orc, seed, M, N, noise=0.3):
    x = _c64(wl.unit_phasors(seed, M, N))
    h = _c64(orc.project(x.astype(np.complex128) + noise * wl.complex_normal(seed, M, N)))
    return x, h


def _ctx(api, M, N, B, nu, k_lo, k_hi, **kw):
    kw.setdefault("r_n", 100)
    return api.Context(M, N, B, nu, k_lo, k_hi, **kw)


FFT_CASES = [
    # M, N, L, k_lo, k_hi, nu0
    (2, 64, 64, -63, 63, -0.5),       # tiny shape, every delay
    (3, 50, 32, -49, 49, -0.5),       # N > L: products folded modulo L, ragged rows
    (2, 20, 64, -19, 19, -0.5),       # N < L: zero-padded
    (1, 40, 128, -7, 30, 0.0123),     # offset grid, asymmetric window, single waveform
    (2, 300, 512, -299, 299, -0.5),   # several CTAs per pair with a ragged tail
    (2, 200, 1024, -60, 80, -0.5),
    (2, 256, 2048, -255, 255, -0.5),  # named-barrier rows (4 warps per row)
    (1, 64, 4096, -10, 10, -0.5),     # largest transform
    (1, 2, 32, -1, 1, -0.5),          # smallest N
]


@pytest.mark.parametrize("elems", ["8", "16", "32"])
@pytest.mark.parametrize("case", FFT_CASES)
def test_ambiguity_fft_matches_oracle(api, orc, case, elems, monkeypatch):
    """Every register-FFT shape (8, 16 or 32 values per thread; a shape that
    does not fit the row length falls back to the default) against the oracle."""
    monkeypatch.setenv("SQNGD_FFT_E", elems)
    M, N, L, k_lo, k_hi, nu0 = case
    nu = nu0 + np.arange(L) / L
    x, h = _pair(orc, 100 + N, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi)
    assert ctx.path == api.AF_PATH_FFT
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    err = np.max(np.abs(chi - ref))
    assert err <= CHI_TOL * N, err / N


WIDE_CASES = [
    # M, N, L, k_lo, k_hi, nu0: rows of >= 1024 bins, where 512-thread CTAs are built
    (2, 200, 1024, -60, 80, -0.5),
    (2, 256, 2048, -255, 255, -0.5),
    (3, 700, 2048, -699, 699, 0.0017),  # several chunks per pair, ragged tail, offset grid
    (1, 64, 4096, -10, 10, -0.5),
    (2, 2500, 1024, -300, 300, -0.5),  # N > L: folded products, the h window spans 3 L
]


@pytest.mark.parametrize("elems", ["16", "32"])
@pytest.mark.parametrize("case", WIDE_CASES)
def test_ambiguity_fft_512_thread_ctas(api, orc, case, elems, monkeypatch):
    """512-thread CTAs (eight or four rows per step sharing x, the h window
    and the twiddles) against the oracle: the grid and the fused maxima."""
    monkeypatch.setenv("SQNGD_FFT_E", elems)
    monkeypatch.setenv("SQNGD_FFT_NT", "512")
    M, N, L, k_lo, k_hi, nu0 = case
    nu = nu0 + np.arange(L) / L
    x, h = _pair(orc, 300 + N, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi)
    assert ctx.path == api.AF_PATH_FFT
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    assert np.max(np.abs(chi - ref)) <= CHI_TOL * N
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h))
    ctx.af_sync()
    t = terms.cpu().numpy()
    r = orc.loss(x, h, nu, k_lo, k_hi)
    for gi, key in ((2, "wapsl"), (3, "wcpsl")):
        if r[key] > 0:
            assert abs(20 * np.log10(t[gi] / r[key])) <= DB_TOL, key
        else:
            assert t[gi] == 0.0, key                  # an empty class (one waveform: no cross pairs)


DFT_CASES = [
    # M, N, nu, k_lo, k_hi
    (2, 100, wl.window_grid(0.05, 64), -40, 40),
    (3, 64, wl.window_grid(0.1, 100), -63, 63),
    (1, 200, np.sort(wl.uniform(5, 37, 1) - 0.5), -20, 20),
    (2, 130, np.array([0.0]), -129, 129),            # zero-Doppler correlation row
]


@pytest.mark.parametrize("case", DFT_CASES)
def test_ambiguity_dft_matches_oracle(api, orc, case):
    M, N, nu, k_lo, k_hi = case
    x, h = _pair(orc, 200 + N, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi)
    assert ctx.path == api.AF_PATH_DFT
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    assert np.max(np.abs(chi - ref)) <= CHI_TOL * N


def _check_terms(orc, api, ctx, x, h, nu, k_lo, k_hi, eps, snrl_db, weights=None):
    M, N = x.shape
    gx = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h), grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    r = orc.loss(x, h, nu, k_lo, k_hi, weights=weights, eps=eps, snrl_db=snrl_db)
    # loss terms
    for gi, key in ((2, "wapsl"), (3, "wcpsl")):
        assert abs(t[gi] - r[key]) <= CHI_TOL, (key, t[gi], r[key])
        if r[key] > 0:
            assert abs(20 * np.log10(t[gi] / r[key])) <= DB_TOL
    np.testing.assert_allclose(t[8:8 + M], r["p"], atol=1e-6)
    assert abs(t[4] - r["snrl_term"]) <= 1e-6
    assert abs(t[0] - r["loss"]) <= CHI_TOL
    # the GPU's winning cell is a max of the oracle's grid within the FP32 bound
    cls = int(t[5])
    cell = int(t[6 + cls])
    assert cell >= 0
    full = orc.ambiguity(x, h, nu, k_lo, k_hi).reshape(-1)
    D, L = k_hi - k_lo + 1, nu.size
    d, j = (cell // L) % D, cell % L
    w = (1.0 / N) if weights is None else weights[d, j]
    assert w * abs(full[cell]) >= r["wpsl"] - CHI_TOL
    # gradient = the oracle's analytic gradient at that cell
    _, ogx, ogh = orc.grad_xh(x, h, nu, k_lo, k_hi, weights=weights, eps=eps, snrl_db=snrl_db, use_cell=cell)
    scale = max(np.max(np.abs(ogx)), np.max(np.abs(ogh)))
    assert np.max(np.abs(gx.cpu().numpy() - ogx)) <= 1e-4 * scale
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 1e-4 * scale
    return t, r


@pytest.mark.parametrize("case", [FFT_CASES[0], FFT_CASES[1], FFT_CASES[4], FFT_CASES[3]])
def test_loss_and_gradient_fft(api, orc, case):
    M, N, L, k_lo, k_hi, nu0 = case
    nu = nu0 + np.arange(L) / L
    x, h = _pair(orc, 300 + N, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5)
    _check_terms(orc, api, ctx, x, h, nu, k_lo, k_hi, 0.3, 0.5)


@pytest.mark.parametrize("case", DFT_CASES[:3])
def test_loss_and_gradient_dft(api, orc, case):
    M, N, nu, k_lo, k_hi = case
    x, h = _pair(orc, 400 + N, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi, eps=0.2, snrl_db=1.0)
    _check_terms(orc, api, ctx, x, h, nu, k_lo, k_hi, 0.2, 1.0)


@pytest.mark.parametrize("M,N,L,k_lo,k_hi", [
    (2, 48, 64, -47, 47),
    (2, 160, 2048, -60, 70),     # 2048-bin rows: the paired last pass of the 32-value transform
])
def test_loss_with_weight_map(api, orc, M, N, L, k_lo, k_hi):
    nu = wl.full_grid(L)
    D = k_hi - k_lo + 1
    wts = (wl.uniform(9, D * L, 3).reshape(D, L) / N).astype(np.float32)
    wts[:, :5] = 0.0                      # cells outside the ROI
    wts = wts.astype(np.float64)
    x, h = _pair(orc, 9, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi, weights=wts, eps=0.5)
    _check_terms(orc, api, ctx, x, h, nu, k_lo, k_hi, 0.5, 0.5, weights=wts)


def test_single_waveform_has_no_cross_term(api, orc):
    N, L = 40, 32
    nu = wl.full_grid(L)
    x, h = _pair(orc, 10, 1, N)
    ctx = _ctx(api, 1, N, 4, nu, -(N - 1), N - 1)
    t, r = _check_terms(orc, api, ctx, x, h, nu, -(N - 1), N - 1, 0.1, 0.5)
    assert t[3] == 0.0 and t[7] == -1 and t[5] == 0


def test_window_without_auto_cells(api, orc):
    """Delay window {0}: the auto class is empty, the cross class carries the loss."""
    M, N, L = 2, 32, 32
    nu = wl.full_grid(L)
    x, h = _pair(orc, 11, M, N)
    ctx = _ctx(api, M, N, 4, nu, 0, 0)
    t, r = _check_terms(orc, api, ctx, x, h, nu, 0, 0, 0.1, 0.5)
    assert t[2] == 0.0 and t[6] == -1 and t[5] == 1


def test_loss_grad_through_soft_chain(api, orc):
    M, N, L, B, r_n, c = 2, 64, 64, 4, 100, 300.0
    nu = wl.full_grid(L)
    u = (wl.logits(12, M, N, 1.5)).astype(np.float32)
    _, h = _pair(orc, 12, M, N)
    ctx = _ctx(api, M, N, B, nu, -(N - 1), N - 1, r_n=r_n, c=c, eps=0.25)
    gu = torch.empty((M, N), dtype=torch.float32, device="cuda")
    gh = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    terms, _, _ = ctx.af_loss_grad(_dev(u), _dev(h), use_hard=False, grad_u=gu, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    rho, a = orc.thresholds(B, r_n)
    rho = rho.astype(np.float32).astype(np.float64)
    cell = int(t[6 + int(t[5])])
    ot, ogu, ogh = orc.loss_grad_u(u.astype(np.float64), h, rho, a, c, nu, -(N - 1), N - 1, eps=0.25,
                                  use_cell=cell)
    assert abs(t[0] - ot[0]) <= 1e-4
    assert np.max(np.abs(gu.cpu().numpy() - ogu)) <= 2e-3 * np.max(np.abs(ogu))
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 1e-3 * np.max(np.abs(ogh))


def test_autograd_function_returns_library_gradient(api, orc):
    M, N, L = 2, 32, 32
    nu = wl.full_grid(L)
    ctx = _ctx(api, M, N, 4, nu, -(N - 1), N - 1, r_n=10)
    u = _dev(wl.logits(13, M, N).astype(np.float32)).requires_grad_(True)
    _, h0 = _pair(orc, 13, M, N)
    h = _dev(h0).requires_grad_(True)
    loss = api.AfLoss.apply(u, h, ctx)
    (2.0 * loss).backward()
    gu = torch.empty((M, N), dtype=torch.float32, device="cuda")
    gh = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    ctx.af_loss_grad(u.detach(), h.detach(), grad_u=gu, grad_h=gh)
    torch.testing.assert_close(u.grad, 2 * gu)
    torch.testing.assert_close(h.grad, 2 * gh)


# ------------------------------------------------------------------ quantizers
@pytest.mark.parametrize("B,r_n", [(4, 3), (16, 100), (64, 100), (8, 1)])
def test_quantize_bit_exact(api, orc, B, r_n):
    rho, _ = orc.thresholds(B, r_n)
    rho32 = rho.astype(np.float32)
    z = wl.uniform(B, 20000, 1).astype(np.float32)
    edge = np.concatenate([rho32, np.nextafter(rho32, np.float32(0)), np.nextafter(rho32, np.float32(1)),
                           np.array([0.0, 1.0], dtype=np.float32)])
    z = np.concatenate([z, edge]).astype(np.float32)
    ctx = _ctx(api, 1, 8, B, wl.full_grid(32), -7, 7, r_n=r_n)
    q, x = ctx.quantize(_dev(z))
    ctx.af_sync()
    oq, ob = orc.hard_quantize(z.astype(np.float64), rho32.astype(np.float64), B)
    np.testing.assert_array_equal(q.cpu().numpy(), oq)
    np.testing.assert_allclose(x.cpu().numpy(), np.exp(2j * np.pi * ob / B), atol=2e-7)


@pytest.mark.parametrize("B,r_n,c", [
    (16, 100, 300.0),    # K = 1600: closed form (alpha = 2c/K = 3/8)
    (64, 100, 300.0),    # K = 6400: closed form (alpha = 3/32)
    (8, 100, 100.0),     # closed form at alpha = 1/4
    (4, 100, 300.0),     # alpha = 3/2: the windowed sum
    (8, 100, 300.0),     # alpha = 3/4: the windowed sum
])
def test_soft_quantize_matches_oracle(api, orc, B, r_n, c):
    """Eq. 24 against the oracle's sum of all K terms, on random z and on the
    ends of [0, 1] where the sum is not saturated on one side."""
    rho, a = orc.thresholds(B, r_n)
    rho32 = rho.astype(np.float32).astype(np.float64)
    u = wl.uniform(21, 5000, 2)
    z = np.concatenate([u[:4000], 0.03 * u[4000:4500], 1.0 - 0.03 * u[4500:], [0.0, 1.0, 1e-6, 1.0 - 1e-6]])
    z = z.astype(np.float32)
    ctx = _ctx(api, 1, 8, B, wl.full_grid(32), -7, 7, r_n=r_n, c=c)
    y, dy, x = ctx.soft_quantize(_dev(z))
    ctx.af_sync()
    oy, ody = orc.soft_quantize(z.astype(np.float64), rho32, a, c)
    assert np.max(np.abs(y.cpu().numpy() - oy)) <= 2e-5
    np.testing.assert_allclose(dy.cpu().numpy(), ody, rtol=1e-4, atol=1e-4)
    assert np.max(np.abs(x.cpu().numpy() - np.exp(2j * np.pi * oy))) <= 1e-4


def test_projection_energy(api, orc):
    M, N = 5, 777
    h = _c64(3 * wl.complex_normal(22, M, N))
    ctx = _ctx(api, M, N, 4, wl.full_grid(32), -3, 3)
    hd = ctx.af_project(_dev(h))
    ctx.af_sync()
    np.testing.assert_allclose(np.sum(np.abs(hd.cpu().numpy().astype(np.complex128)) ** 2, axis=1), N, rtol=2e-6)
    np.testing.assert_allclose(hd.cpu().numpy(), orc.project(h), rtol=0, atol=2e-6)


def test_init_maps_indices_and_projects(api, orc):
    M, N, B, r_n = 3, 100, 16, 100
    ctx = _ctx(api, M, N, B, wl.full_grid(32), -5, 5, r_n=r_n)
    b = wl.phase_indices(3, M, N, B)
    u, h = ctx.sqngd_init(_dev(b))
    q, _ = ctx.quantize(torch.sigmoid(u))
    ctx.af_sync()
    np.testing.assert_array_equal(q.cpu().numpy() % B, b)
    np.testing.assert_allclose(h.cpu().numpy(), np.exp(2j * np.pi * b / B), atol=2e-6)
    np.testing.assert_allclose(u.cpu().numpy(), orc.init_logits(b, B, r_n), rtol=1e-6)


# ------------------------------------------------------------------ optimiser
def _state(api, u, h):
    return api.SqngdState.create(_dev(u), _dev(h))


def test_adam_step_on_filters_matches_oracle(api, orc):
    M, N, L, B, r_n = 2, 64, 64, 4, 10
    nu = wl.full_grid(L)
    b = wl.phase_indices(5, M, N, B)
    u = orc.init_logits(b, B, r_n).astype(np.float32)
    _, h = _pair(orc, 5, M, N, 0.2)
    ctx = _ctx(api, M, N, B, nu, -(N - 1), N - 1, r_n=r_n, n_h=1, n_x=0, lr_h=0.05)
    gh = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    ctx.af_loss_grad(_dev(u), _dev(h), use_hard=True, grad_h=gh)
    g = gh.cpu().numpy().astype(np.complex128)
    st = _state(api, u, h)
    log = ctx.sqngd_step(st, 1)
    assert st.t_h == 1 and st.t_x == 0 and st.outer == 1
    theta = h.astype(np.complex128).view(np.float64).copy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    orc.adam(theta, g.view(np.float64), m, v, 1, 0.05)
    exp = orc.project(theta.view(np.complex128).reshape(M, N))
    np.testing.assert_allclose(st.h.cpu().numpy(), exp, atol=5e-6)
    assert np.isfinite(log).all()


def test_adam_step_on_logits_matches_oracle(api, orc):
    M, N, L, B, r_n = 2, 64, 64, 4, 10
    nu = wl.full_grid(L)
    u = wl.logits(6, M, N, 1.0).astype(np.float32)
    _, h = _pair(orc, 6, M, N, 0.2)
    ctx = _ctx(api, M, N, B, nu, -(N - 1), N - 1, r_n=r_n, n_h=0, n_x=1, lr_x=1e-3)
    gu = torch.empty((M, N), dtype=torch.float32, device="cuda")
    ctx.af_loss_grad(_dev(u), _dev(h), use_hard=False, grad_u=gu)
    g = gu.cpu().numpy().astype(np.float64)
    st = _state(api, u, h)
    ctx.sqngd_step(st, 1)
    theta = u.astype(np.float64).copy()
    orc.adam(theta, g, np.zeros_like(theta), np.zeros_like(theta), 1, 1e-3)
    np.testing.assert_allclose(st.u.cpu().numpy(), theta, atol=2e-6)
    np.testing.assert_array_equal(st.h.cpu().numpy(), h)


def test_eval_hard_fp64_matches_oracle(api, orc):
    for (M, N, nu, k_lo, k_hi) in ((2, 64, wl.full_grid(64), -63, 63), (2, 90, wl.window_grid(0.05, 40), -30, 30)):
        B, r_n = 4, 10
        b = wl.phase_indices(7, M, N, B)
        u = orc.init_logits(b, B, r_n).astype(np.float32)
        _, h = _pair(orc, 7, M, N, 0.2)
        ctx = _ctx(api, M, N, B, nu, k_lo, k_hi, r_n=r_n)
        out = ctx.af_eval_hard(_dev(u), _dev(h))
        x = np.exp(2j * np.pi * b / B)
        met, snrl = orc.metrics(x, h, nu, k_lo, k_hi)
        np.testing.assert_allclose(out[:4], met, atol=1e-8)
        np.testing.assert_allclose(out[4:], snrl, atol=1e-8)


def test_nonfinite_filter_is_reported(api, orc):
    M, N = 1, 32
    ctx = _ctx(api, M, N, 4, wl.full_grid(32), -31, 31)
    x, h = _pair(orc, 14, M, N)
    h[0, 3] = np.nan
    ctx.af_loss_grad_xh(_dev(x), _dev(h))
    with pytest.raises(api.AfError, match="AF_ERR_NONFINITE"):
        ctx.af_sync()
    ctx.af_sync()   # the flag is cleared once reported


# ------------------------------------------------------------------ full sizes
def _sampled_cells(seed, total, n=3000):
    return np.unique((wl.uniform(seed, n, 4) * total).astype(np.int64))


@pytest.mark.parametrize("which", ["mid", "differentiation", "precision"])
def test_full_size_sampled_cells(api, orc, which):
    w = getattr(wl, which)()
    x, h = _pair(orc, 31, w.M, w.N)
    ctx = _ctx(api, w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi)
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).reshape(-1)
    cells = _sampled_cells(31, chi.numel())
    got = chi[torch.from_numpy(cells).cuda()].cpu().numpy()
    ref = orc.ambiguity_cells(x, h, w.nu, w.k_lo, w.k_hi, cells)
    assert np.max(np.abs(got - ref)) <= CHI_TOL * w.N


def test_full_size_mid_loss_matches_oracle(api, orc):
    """The launch configuration the benchmark times (M=4, N=512, 512 bins)."""
    w = wl.mid()
    x, h = _pair(orc, 32, w.M, w.N)
    ctx = _ctx(api, w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db)
    _check_terms(orc, api, ctx, x, h, w.nu, w.k_lo, w.k_hi, w.eps, w.snrl_db)


def test_full_size_differentiation_max_and_gradient(api, orc):
    """M=4, N=2048, 2048 bins: the reported max is the oracle's value at that
    cell, no sampled cell exceeds it, and the gradient is the oracle's at it."""
    w = wl.differentiation()
    x, h = _pair(orc, 33, w.M, w.N)
    ctx = _ctx(api, w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db)
    gx = torch.empty((w.M, w.N), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h), grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    cell = int(t[6 + int(t[5])])
    chi, ogx, ogh = orc.grad_at_cell(x, h, w.nu, w.k_lo, w.k_hi, cell, 1.0 / w.N, eps=w.eps, snrl_db=w.snrl_db)
    assert abs(abs(chi) / w.N - t[1]) <= CHI_TOL
    cells = _sampled_cells(33, w.M * w.M * w.D * w.L, 20000)
    D, L = w.D, w.L
    pair = cells // (D * L)
    k = (cells // L) % D + w.k_lo
    keep = ~((pair // w.M == pair % w.M) & (k == 0))
    vals = np.abs(orc.ambiguity_cells(x, h, w.nu, w.k_lo, w.k_hi, cells[keep])) / w.N
    assert vals.max() <= t[1] + CHI_TOL
    scale = max(np.max(np.abs(ogx)), np.max(np.abs(ogh)))
    assert np.max(np.abs(gx.cpu().numpy() - ogx)) <= 1e-4 * scale
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 1e-4 * scale


# ------------------------------------------------------------------ Algorithm 1
def test_sqngd_tiny_run_tracks_oracle_statistically(api, orc):
    """200 outer iterations of the tiny problem from 5 seeds: trajectories
    diverge (max switches), so the final hard PSLR medians are compared."""
    w = wl.tiny()
    rho, a = orc.thresholds(w.B, w.r_n)
    rho32 = rho.astype(np.float32).astype(np.float64)
    n_outer = 200
    g_final, o_final = [], []
    for seed in range(5):
        b = wl.phase_indices(seed, w.M, w.N, w.B)
        u0 = orc.init_logits(b, w.B, w.r_n).astype(np.float32)
        h0 = _c64(orc.project(np.exp(2j * np.pi * b / w.B)))
        ctx = _ctx(api, w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db,
                   lr_h=w.lr_h, lr_x=w.lr_x)
        st = _state(api, u0, h0)
        log = ctx.sqngd_step(st, n_outer)
        assert np.isfinite(log).all()
        best = st.best.cpu().numpy()
        out = ctx.af_eval_hard(st.u, st.h)
        g_final.append(out[2])
        assert best[0] < np.inf
        # oracle run of the same length from the same start
        ost = dict(u=u0.astype(np.float64), h=h0.astype(np.complex128), mu=np.zeros((w.M, w.N)),
                   vu=np.zeros((w.M, w.N)), mh=np.zeros((w.M, w.N), complex), vh=np.zeros((w.M, w.N), complex),
                   t_x=0, t_h=0)
        cfg = dict(nu=w.nu, k_lo=w.k_lo, k_hi=w.k_hi, eps=w.eps, snrl_db=w.snrl_db, B=w.B, rho=rho32, a=a,
                   c=w.c, n_h=w.n_h, n_x=w.n_x, lr_h=w.lr_h, lr_x=w.lr_x)
        for _ in range(n_outer):
            orc.sqngd_outer(ost, cfg)
        _, xo = orc.hard_waveform(ost["u"], rho32, w.B)
        met, _ = orc.metrics(xo, ost["h"], w.nu, w.k_lo, w.k_hi)
        o_final.append(met[2])
        # both runs improved on the start
        start, _ = orc.metrics(np.exp(2j * np.pi * b / w.B), h0, w.nu, w.k_lo, w.k_hi)
        assert out[2] < start[2] and met[2] < start[2]
    assert abs(np.median(g_final) - np.median(o_final)) <= 0.5, (g_final, o_final)


def test_quantize_with_user_thresholds_bit_exact(api, orc):
    """Non-uniform thresholds (af_set_thresholds) take the binary-search path."""
    B, r_n = 8, 5
    K = B * r_n
    rho = np.sort(wl.uniform(23, K, 1)).astype(np.float32)
    z = np.concatenate([wl.uniform(24, 5000, 1).astype(np.float32), rho,
                        np.nextafter(rho, np.float32(0))]).astype(np.float32)
    ctx = _ctx(api, 1, 8, B, wl.full_grid(32), -7, 7, r_n=r_n)
    ctx.af_set_thresholds(rho)
    q, _ = ctx.quantize(_dev(z))
    y, dy, _ = ctx.soft_quantize(_dev(z))
    ctx.af_sync()
    oq, _ = orc.hard_quantize(z.astype(np.float64), rho.astype(np.float64), B)
    np.testing.assert_array_equal(q.cpu().numpy(), oq)
    oy, ody = orc.soft_quantize(z.astype(np.float64), rho.astype(np.float64), 1.0 / (2 * B), 300.0)
    assert np.max(np.abs(y.cpu().numpy() - oy)) <= 2e-5


# ------------------------------------------------------------------ p-norm, dense adjoint
PNORM_CASES = [
    # M, N, L, k_lo, k_hi
    (2, 64, 64, -63, 63),
    (3, 50, 32, -30, 49),       # folded products, asymmetric window
    (2, 200, 256, -199, 199),   # several CTAs per pair
    (1, 40, 128, -39, 39),      # single waveform: auto class only
]


@pytest.mark.parametrize("elems", ["8", "16"])
@pytest.mark.parametrize("pn", [5.0, 8.0, 16.0])
@pytest.mark.parametrize("case", PNORM_CASES)
def test_pnorm_loss_and_dense_gradient(api, orc, case, pn, elems, monkeypatch):
    """Smooth p-norm sidelobe loss: every cell of the winning class carries
    gradient, recomputed by the dense adjoint; compared with the oracle's
    analytic gradient (unique, no tie choice)."""
    monkeypatch.setenv("SQNGD_FFT_E", elems)
    M, N, L, k_lo, k_hi = case
    nu = wl.full_grid(L)
    x, h = _pair(orc, 500 + N, M, N)
    ctx = _ctx(api, M, N, 4, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5, pnorm=pn)
    gx = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h), grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    ot, ogx, ogh = orc.grad_xh(x, h, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5, pnorm=pn)
    np.testing.assert_allclose(t[[0, 2, 3, 4]], ot[[0, 2, 3, 4]], rtol=2e-5, atol=1e-6)
    assert int(t[5]) == int(ot[5])
    scale = max(np.max(np.abs(ogx)), np.max(np.abs(ogh)))
    assert np.max(np.abs(gx.cpu().numpy() - ogx)) <= 2e-4 * scale
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 2e-4 * scale


def test_pnorm_with_weight_map_and_soft_chain(api, orc):
    M, N, L = 2, 48, 64
    nu = wl.full_grid(L)
    k_lo, k_hi = -47, 47
    D = k_hi - k_lo + 1
    wts = (wl.uniform(19, D * L, 3).reshape(D, L) / N).astype(np.float32)
    wts[:10, :] = 0.0
    wts = wts.astype(np.float64)
    B, r_n, c = 4, 10, 300.0
    u = wl.logits(19, M, N, 1.0).astype(np.float32)
    _, h = _pair(orc, 19, M, N)
    ctx = _ctx(api, M, N, B, nu, k_lo, k_hi, weights=wts, eps=0.4, r_n=r_n, c=c, pnorm=8.0)
    gu = torch.empty((M, N), dtype=torch.float32, device="cuda")
    gh = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    terms, _, _ = ctx.af_loss_grad(_dev(u), _dev(h), use_hard=False, grad_u=gu, grad_h=gh)
    ctx.af_sync()
    rho, a = orc.thresholds(B, r_n)
    rho = rho.astype(np.float32).astype(np.float64)
    ot, ogu, ogh = orc.loss_grad_u(u.astype(np.float64), h, rho, a, c, nu, k_lo, k_hi, weights=wts, eps=0.4,
                                  pnorm=8.0)
    assert abs(terms.cpu().numpy()[0] - ot[0]) <= 1e-4 * max(1.0, abs(ot[0]))
    assert np.max(np.abs(gu.cpu().numpy() - ogu)) <= 2e-3 * np.max(np.abs(ogu))
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 1e-3 * np.max(np.abs(ogh))


def test_pnorm_optimiser_runs(api, orc):
    w = wl.tiny()
    b = wl.phase_indices(3, w.M, w.N, w.B)
    ctx = _ctx(api, w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, r_n=w.r_n, pnorm=16.0, lr_h=w.lr_h, lr_x=w.lr_x)
    u, h = ctx.sqngd_init(_dev(b))
    st = api.SqngdState.create(u, h)
    log = ctx.sqngd_step(st, 20)
    assert np.isfinite(log).all()
    assert log[-1, 0, 0] < log[0, 0, 0]


@pytest.mark.parametrize("pn", [0.0, 8.0])
def test_full_size_differentiation_gradient_invariants(api, orc, pn):
    """M=4, N=2048, 2048 bins, exact max and dense p-norm adjoint: with eps = 1
    the loss is 1-homogeneous in h and in x (Re<grad, v> = L_WPSL) and
    invariant to a common phase rotation of any x_m or h_l."""
    w = wl.differentiation()
    x, h = _pair(orc, 34, w.M, w.N)
    ctx = _ctx(api, w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=1.0, snrl_db=w.snrl_db, pnorm=pn)
    gx = torch.empty((w.M, w.N), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h), grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    gxn = gx.cpu().numpy().astype(np.complex128)
    ghn = gh.cpu().numpy().astype(np.complex128)
    xn, hn = x.astype(np.complex128), h.astype(np.complex128)
    assert abs(np.sum(np.real(np.conj(ghn) * hn)) - t[1]) <= 1e-4 * t[1]
    assert abs(np.sum(np.real(np.conj(gxn) * xn)) - t[1]) <= 1e-4 * t[1]
    scale = np.sum(np.abs(gxn) * np.abs(xn), axis=1).max()
    for m in range(w.M):
        assert abs(np.sum(np.imag(np.conj(xn[m]) * gxn[m]))) <= 1e-4 * scale
        assert abs(np.sum(np.real(np.conj(ghn[m]) * 1j * hn[m]))) <= 1e-4 * scale
    if pn > 0:
        # every waveform row carries dense gradient, not one cell's worth
        assert np.count_nonzero(np.abs(gxn) > 1e-3 * np.abs(gxn).max()) > w.M * w.N // 2


def test_pnorm_on_arbitrary_grid_is_unimplemented(api):
    with pytest.raises(api.AfError, match="AF_ERR_UNIMPLEMENTED"):
        api.Context(2, 64, 4, wl.window_grid(0.05, 40), -10, 10, pnorm=8.0)
