"""Trainable quantization thresholds (Section III-C, Eq. 24 with rho trained in
Step B of Algorithm 1) against the FP64 oracle, through the C ABI: dL/drho,
the projection onto the ordered set in [0, 1], one outer iteration and a
100-iteration run compared statistically."""
import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import api as a
    return a


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _h(orc, seed, M, N):
    return orc.project(wl.unit_phasors(seed, M, N) + 0.2 * wl.complex_normal(seed, M, N)).astype(np.complex64)


@pytest.mark.parametrize("r_n,c", [(100, 300.0), (3, 40.0)])
def test_threshold_gradient_matches_oracle(api, orc, r_n, c):
    M, N, L, B = 2, 64, 64, 4
    nu = wl.full_grid(L)
    u = wl.logits(51, M, N, 1.5).astype(np.float32)
    h = _h(orc, 51, M, N)
    ctx = api.Context(M, N, B, nu, -(N - 1), N - 1, eps=0.25, r_n=r_n, c=c, n_h=0, n_x=1, train_rho=True)
    gu = torch.empty((M, N), dtype=torch.float32, device="cuda")
    terms, _, _, gr = ctx.af_loss_grad_rho(_dev(u), _dev(h), grad_u=gu)
    ctx.af_sync()
    t = terms.cpu().numpy()
    rho, a = orc.thresholds(B, r_n)
    rho = rho.astype(np.float32).astype(np.float64)
    cell = int(t[6 + int(t[5])])
    ot, ogu, ogr = orc.loss_grad_u_rho(u.astype(np.float64), h, rho, a, c, nu, -(N - 1), N - 1, eps=0.25,
                                       use_cell=cell)
    assert abs(t[0] - ot[0]) <= 1e-4
    assert np.max(np.abs(gu.cpu().numpy() - ogu)) <= 2e-3 * np.max(np.abs(ogu))
    g = gr.cpu().numpy()
    assert np.max(np.abs(g - ogr)) <= 2e-3 * np.max(np.abs(ogr)), np.max(np.abs(g - ogr)) / np.max(np.abs(ogr))
    ctx.close()


@pytest.mark.parametrize("B,r_n", [(4, 100), (37, 1)])
def test_projection_matches_oracle(api, orc, B, r_n):
    K = B * r_n
    ctx = api.Context(2, 32, B, wl.full_grid(32), -31, 31, r_n=r_n, n_h=0, n_x=1, train_rho=True)
    base, _ = orc.thresholds(B, r_n)
    for seed in range(3):
        r = (base + (wl.uniform(60 + seed, K, 1) - 0.5) * (4.0 / K) * (1 + 10 * seed)).astype(np.float32)
        r[:2] -= 0.01 * seed                                  # a few below 0 at larger perturbations
        got = ctx.af_project_thresholds(_dev(r)).cpu().numpy()
        exp = orc.project_thresholds(r.astype(np.float64))
        np.testing.assert_allclose(got, exp, atol=2e-6)
        assert np.all(np.diff(got) >= 0) and got.min() >= 0 and got.max() <= 1
    # an ordered set inside [0, 1] is left as it is
    got = ctx.af_project_thresholds(_dev(base.astype(np.float32))).cpu().numpy()
    np.testing.assert_array_equal(got, base.astype(np.float32))
    ctx.close()


def test_one_outer_iteration_updates_u_and_rho(api, orc):
    """n_h = 0, n_x = 1: one transmit step = Adam on u and on rho with the
    gradients af_loss_grad_rho reports, then the projection."""
    M, N, L, B, r_n, lr_rho = 2, 64, 64, 4, 10, 2e-3
    nu = wl.full_grid(L)
    u = wl.logits(52, M, N, 1.0).astype(np.float32)
    h = _h(orc, 52, M, N)
    ctx = api.Context(M, N, B, nu, -(N - 1), N - 1, r_n=r_n, n_h=0, n_x=1, lr_x=1e-3, train_rho=True,
                      lr_rho=lr_rho)
    rho0 = ctx.af_get_thresholds().astype(np.float64)
    gu = torch.empty((M, N), dtype=torch.float32, device="cuda")
    _, _, _, gr = ctx.af_loss_grad_rho(_dev(u), _dev(h), grad_u=gu)
    g_u = gu.cpu().numpy().astype(np.float64)
    g_r = gr.cpu().numpy().astype(np.float64)
    st = api.SqngdState.create(_dev(u), _dev(h))
    log = ctx.sqngd_step(st, 1)
    assert np.isfinite(log).all()
    theta = u.astype(np.float64).copy()
    orc.adam(theta, g_u, np.zeros_like(theta), np.zeros_like(theta), 1, 1e-3)
    np.testing.assert_allclose(st.u.cpu().numpy(), theta, atol=2e-6)
    r = rho0.copy()
    orc.adam(r, g_r, np.zeros_like(r), np.zeros_like(r), 1, lr_rho)
    exp = orc.project_thresholds(r)
    got = ctx.af_get_thresholds()
    np.testing.assert_allclose(got, exp, atol=2e-6)
    assert not np.array_equal(got, rho0.astype(np.float32))
    ctx.close()


def test_trained_thresholds_run_tracks_oracle_statistically(api, orc):
    """100 outer iterations of the tiny problem (r_n = 10) from 3 seeds with
    trained thresholds: thresholds stay ordered in [0, 1] and move; the final
    hard PSLR medians of GPU and oracle agree within 0.5 dB."""
    w = wl.tiny()
    r_n, lr_rho, n_outer = 10, 1e-4, 100
    rho, a = orc.thresholds(w.B, r_n)
    rho32 = rho.astype(np.float32).astype(np.float64)
    g_final, o_final = [], []
    for seed in range(3):
        b = wl.phase_indices(seed, w.M, w.N, w.B)
        u0 = orc.init_logits(b, w.B, r_n).astype(np.float32)
        h0 = orc.project(np.exp(2j * np.pi * b / w.B)).astype(np.complex64)
        ctx = api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db, r_n=r_n, c=w.c,
                          lr_h=w.lr_h, lr_x=w.lr_x, train_rho=True, lr_rho=lr_rho)
        st = api.SqngdState.create(_dev(u0), _dev(h0))
        log = ctx.sqngd_step(st, n_outer)
        assert np.isfinite(log).all()
        rg = ctx.af_get_thresholds()
        assert np.all(np.diff(rg) >= 0) and rg.min() >= 0 and rg.max() <= 1
        assert np.max(np.abs(rg - rho32)) > 0
        out = ctx.af_eval_hard(st.u, st.h)
        g_final.append(out[2])
        ctx.close()
        ost = dict(u=u0.astype(np.float64), h=h0.astype(np.complex128), mu=np.zeros((w.M, w.N)),
                   vu=np.zeros((w.M, w.N)), mh=np.zeros((w.M, w.N), complex), vh=np.zeros((w.M, w.N), complex),
                   rho=rho32.copy(), mr=np.zeros_like(rho32), vr=np.zeros_like(rho32), t_x=0, t_h=0)
        cfg = dict(nu=w.nu, k_lo=w.k_lo, k_hi=w.k_hi, eps=w.eps, snrl_db=w.snrl_db, B=w.B, a=a, c=w.c,
                   n_h=w.n_h, n_x=w.n_x, lr_h=w.lr_h, lr_x=w.lr_x, lr_rho=lr_rho)
        for _ in range(n_outer):
            orc.sqngd_outer_rho(ost, cfg)
        _, xo = orc.hard_waveform(ost["u"], ost["rho"], w.B)
        met, _ = orc.metrics(xo, ost["h"], w.nu, w.k_lo, w.k_hi)
        o_final.append(met[2])
    assert abs(np.median(g_final) - np.median(o_final)) <= 0.5, (g_final, o_final)
