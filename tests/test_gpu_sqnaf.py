"""SQNAF (Section IV): every receive filter is its waveform, h = x.

GPU matched contexts against the oracle's matched functions, through the C
ABI: loss terms of L(x, x), the total gradient (transmit and filter partials
summed) at the GPU's winning cell, the soft chain, the FP64 acceptance pass,
one outer iteration (hard-design score, then Adam on u) and a 200-iteration
run compared statistically.  With h = x the ambiguity function has mirror
ties (|chi_ml(k, nu)| = |chi_lm(-k, -nu)|), so the GPU may pick either cell
of a tied pair: the tests check that its cell attains the oracle's max and
compare the gradient at that cell.
"""
import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CHI_TOL = 1e-5
DB_TOL = 0.05


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import api as a
    return a


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    # M, N, nu, k_lo, k_hi, path, |chi| tolerance scale
    (2, 64, wl.full_grid(64), -63, 63, "fft", 1.0),             # symmetric: mirror ties
    (3, 50, 0.0123 + np.arange(32) / 32, -10, 30, "fft", 1.0),  # offset grid, asymmetric window
    (2, 300, wl.full_grid(512), -299, 299, "fft", 1.0),         # several CTAs per pair
    (2, 90, wl.window_grid(0.05, 40), -30, 30, "dft", 1.0),
    (2, 130, np.array([0.0]), -129, 129, "dft", 1.0),           # zero-Doppler correlation row
    (2, 200, wl.window_grid(0.05, 64), -100, 100, "split", 10.0),
]


@pytest.mark.parametrize("case", CASES)
def test_matched_loss_and_gradient(api, orc, case):
    M, N, nu, k_lo, k_hi, path, tol = case
    p = {"fft": api.AF_PATH_FFT, "dft": api.AF_PATH_DFT, "split": api.AF_PATH_SPLIT_BF16}[path]
    # non-unimodular waveforms so that the SNRL term is not constant
    x = (wl.unit_phasors(500 + N, M, N) + 0.3 * wl.complex_normal(500 + N, M, N)).astype(np.complex64)
    ctx = api.Context(M, N, 4, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5, r_n=10, n_h=0, n_x=10,
                      matched=True, path=p)
    gx = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), None, grad_x=gx)
    ctx.af_sync()
    t = terms.cpu().numpy()
    r = orc.loss(x, x, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5)
    db_tol = 0.1 if path == "split" else DB_TOL
    for gi, key in ((2, "wapsl"), (3, "wcpsl")):
        assert abs(t[gi] - r[key]) <= tol * CHI_TOL, (key, t[gi], r[key])
        if r[key] > 0:
            assert abs(20 * np.log10(t[gi] / r[key])) <= db_tol
    np.testing.assert_allclose(t[8:8 + M], r["p"], atol=1e-6)
    assert abs(t[4] - r["snrl_term"]) <= 1e-6
    cell = int(t[6 + int(t[5])])
    full = orc.ambiguity(x, x, nu, k_lo, k_hi).reshape(-1)
    assert abs(full[cell]) / N >= r["wpsl"] - tol * CHI_TOL
    _, og = orc.grad_matched(x, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5, use_cell=cell)
    assert np.max(np.abs(gx.cpu().numpy() - og)) <= 1e-4 * np.max(np.abs(og))
    ctx.close()


def test_matched_soft_chain(api, orc):
    M, N, L, B, r_n, c = 2, 64, 64, 4, 100, 300.0
    nu = 0.007 + np.arange(L) / L
    k_lo, k_hi = -20, 40
    u = wl.logits(31, M, N, 1.5).astype(np.float32)
    ctx = api.Context(M, N, B, nu, k_lo, k_hi, eps=0.25, r_n=r_n, c=c, n_h=0, n_x=10, matched=True)
    gu = torch.empty((M, N), dtype=torch.float32, device="cuda")
    terms, _, _ = ctx.af_loss_grad(_dev(u), None, use_hard=False, grad_u=gu)
    ctx.af_sync()
    t = terms.cpu().numpy()
    rho, a = orc.thresholds(B, r_n)
    rho = rho.astype(np.float32).astype(np.float64)
    cell = int(t[6 + int(t[5])])
    ot, ogu = orc.loss_grad_u_matched(u.astype(np.float64), rho, a, c, nu, k_lo, k_hi, eps=0.25,
                                      use_cell=cell)
    assert abs(t[0] - ot[0]) <= 1e-4
    assert np.max(np.abs(gu.cpu().numpy() - ogu)) <= 2e-3 * np.max(np.abs(ogu))
    ctx.close()


def test_matched_rejects_filter_gradient(api):
    M, N = 2, 32
    ctx = api.Context(M, N, 4, wl.full_grid(32), -31, 31, n_h=0, n_x=1, matched=True)
    x = _dev(wl.unit_phasors(1, M, N).astype(np.complex64))
    gh = torch.empty_like(x)
    with pytest.raises(api.AfError):
        ctx.af_loss_grad_xh(x, None, grad_h=gh)
    ctx.close()


def test_matched_eval_hard_fp64(api, orc):
    M, N, B, r_n = 2, 90, 4, 10
    nu, k_lo, k_hi = wl.window_grid(0.05, 40), -30, 30
    b = wl.phase_indices(8, M, N, B)
    u = orc.init_logits(b, B, r_n).astype(np.float32)
    ctx = api.Context(M, N, B, nu, k_lo, k_hi, r_n=r_n, n_h=0, n_x=1, matched=True)
    out = ctx.af_eval_hard(_dev(u), None)
    x = np.exp(2j * np.pi * b / B)
    met, snrl = orc.metrics(x, x, nu, k_lo, k_hi)
    np.testing.assert_allclose(out[:4], met, atol=1e-8)
    np.testing.assert_allclose(out[4:], snrl, atol=1e-8)
    assert np.max(np.abs(out[4:])) < 1e-9          # matched filters: SNRL = 0 dB
    ctx.close()


def test_sqnaf_one_outer_iteration(api, orc):
    """Score of the hard design first (best-design record), then one Adam
    step on u with the matched soft-chain gradient; no filter is touched."""
    M, N, L, B, r_n = 2, 64, 64, 4, 10
    nu = wl.full_grid(L)
    u = wl.logits(9, M, N, 1.0).astype(np.float32)
    ctx = api.Context(M, N, B, nu, -(N - 1), N - 1, r_n=r_n, n_h=0, n_x=1, lr_x=1e-3, matched=True)
    gu = torch.empty((M, N), dtype=torch.float32, device="cuda")
    ctx.af_loss_grad(_dev(u), None, use_hard=False, grad_u=gu)
    g = gu.cpu().numpy().astype(np.float64)
    st = api.SqngdState.create(_dev(u))
    log = ctx.sqngd_step(st, 1)
    assert log.shape == (1, 2, 4) and np.isfinite(log).all()
    assert st.t_h == 0 and st.t_x == 1 and st.outer == 1
    theta = u.astype(np.float64).copy()
    orc.adam(theta, g, np.zeros_like(theta), np.zeros_like(theta), 1, 1e-3)
    np.testing.assert_allclose(st.u.cpu().numpy(), theta, atol=2e-6)
    # the score is L(X_hard, X_hard) of the starting logits, and it is the best so far
    rho, _ = orc.thresholds(B, r_n)
    q, xh = orc.hard_waveform(u, rho.astype(np.float32).astype(np.float64), B)
    r = orc.loss(xh, xh, nu, -(N - 1), N - 1)
    assert abs(log[0, 0, 0] - r["loss"]) <= CHI_TOL and abs(log[0, 0, 1] - r["wpsl"]) <= CHI_TOL
    best = st.best.cpu().numpy()
    assert abs(best[0] - r["wpsl"]) <= CHI_TOL and best[2] == 0
    np.testing.assert_array_equal(st.best_q.cpu().numpy(), q)
    np.testing.assert_allclose(st.best_h.cpu().numpy(), xh, atol=1e-6)
    ctx.close()


def test_sqnaf_tiny_run_tracks_oracle_statistically(api, orc):
    """200 SQNAF outer iterations of the tiny problem from 5 seeds against the
    oracle's: the final hard PSLR medians agree within 0.5 dB and both runs
    improve on the start."""
    w = wl.tiny()
    rho, a = orc.thresholds(w.B, w.r_n)
    rho32 = rho.astype(np.float32).astype(np.float64)
    n_outer = 200
    g_final, o_final = [], []
    for seed in range(5):
        b = wl.phase_indices(seed, w.M, w.N, w.B)
        u0 = orc.init_logits(b, w.B, w.r_n).astype(np.float32)
        ctx = api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db, r_n=w.r_n,
                          c=w.c, n_h=0, n_x=w.n_x, lr_x=w.lr_x, matched=True)
        st = api.SqngdState.create(_dev(u0))
        log = ctx.sqngd_step(st, n_outer)
        assert np.isfinite(log).all()
        out = ctx.af_eval_hard(st.u, None)
        g_final.append(out[2])
        ctx.close()
        ost = dict(u=u0.astype(np.float64), mu=np.zeros((w.M, w.N)), vu=np.zeros((w.M, w.N)), t_x=0)
        cfg = dict(nu=w.nu, k_lo=w.k_lo, k_hi=w.k_hi, eps=w.eps, snrl_db=w.snrl_db, B=w.B, rho=rho32, a=a,
                   c=w.c, n_x=w.n_x, lr_x=w.lr_x)
        for _ in range(n_outer):
            orc.sqnaf_outer(ost, cfg)
        _, xo = orc.hard_waveform(ost["u"], rho32, w.B)
        met, _ = orc.metrics(xo, xo, w.nu, w.k_lo, w.k_hi)
        o_final.append(met[2])
        x0 = np.exp(2j * np.pi * b / w.B)
        start, _ = orc.metrics(x0, x0, w.nu, w.k_lo, w.k_hi)
        assert out[2] < start[2] and met[2] < start[2]
    assert abs(np.median(g_final) - np.median(o_final)) <= 0.5, (g_final, o_final)
