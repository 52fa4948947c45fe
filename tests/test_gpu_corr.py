"""Zero-Doppler / single-bin mode (L = 1): the cross-correlation kernel of
the arbitrary-grid path against the FP64 oracle, through the C ABI.

Cases span one and many CTAs per pair (32 delays each), ragged delay
counts, one-sided and single-delay windows, an offset bin nu_0 != 0, the
smallest N, the largest N and the paper's correlation setting (M = 2,
N = 1200, every delay).
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pair(orc, seed, M, N, noise=0.3):
    x = wl.unit_phasors(seed, M, N).astype(np.complex64)
    h = orc.project(x.astype(np.complex128) + noise * wl.complex_normal(seed, M, N)).astype(np.complex64)
    return x, h


CASES = [
    # M, N, nu_0, k_lo, k_hi
    (2, 130, 0.0, -129, 129),
    (2, 1200, 0.0, -1199, 1199),      # the paper's correlation setting
    (1, 2, 0.0, -1, 1),               # smallest N
    (3, 77, 0.013, -50, 20),          # offset bin, asymmetric window, ragged last chunk
    (2, 512, 0.0, 5, 100),            # one-sided window
    (2, 40, 0.0, 0, 0),               # a single delay: the auto class is empty
    (4, 4096, 0.0, -4095, 4095),      # largest N
]


@pytest.mark.parametrize("case", CASES)
def test_corr_ambiguity_matches_oracle(api, orc, case):
    M, N, nu0, k_lo, k_hi = case
    nu = np.array([nu0])
    x, h = _pair(orc, 600 + N, M, N)
    ctx = api.Context(M, N, 4, nu, k_lo, k_hi, r_n=10)
    assert ctx.path == api.AF_PATH_DFT
    chi = ctx.af_ambiguity(_dev(x), _dev(h)).cpu().numpy()
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    assert np.max(np.abs(chi - ref)) <= CHI_TOL * N
    ctx.close()


@pytest.mark.parametrize("case", CASES[:6])
def test_corr_loss_and_gradient(api, orc, case):
    M, N, nu0, k_lo, k_hi = case
    nu = np.array([nu0])
    x, h = _pair(orc, 700 + N, M, N)
    ctx = api.Context(M, N, 4, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5, r_n=10)
    gx = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h), grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    r = orc.loss(x, h, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5)
    for gi, key in ((2, "wapsl"), (3, "wcpsl")):
        assert abs(t[gi] - r[key]) <= CHI_TOL, (key, t[gi], r[key])
        if r[key] > 0:
            assert abs(20 * np.log10(t[gi] / r[key])) <= DB_TOL
    np.testing.assert_allclose(t[8:8 + M], r["p"], atol=1e-6)
    assert abs(t[0] - r["loss"]) <= CHI_TOL
    cls = int(t[5])
    cell = int(t[6 + cls])
    full = orc.ambiguity(x, h, nu, k_lo, k_hi).reshape(-1)
    assert abs(full[cell]) / N >= r["wpsl"] - CHI_TOL
    _, ogx, ogh = orc.grad_xh(x, h, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5, use_cell=cell)
    scale = max(np.max(np.abs(ogx)), np.max(np.abs(ogh)))
    assert np.max(np.abs(gx.cpu().numpy() - ogx)) <= 1e-4 * scale
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 1e-4 * scale
    if k_lo == k_hi == 0:
        assert t[2] == 0.0 and t[6] == -1 and cls == 1
    ctx.close()


def test_corr_weight_map(api, orc):
    """Per-delay weights with some delays outside the ROI."""
    M, N, k_lo, k_hi = 2, 300, -299, 299
    D = k_hi - k_lo + 1
    wts = (wl.uniform(41, D, 3).reshape(D, 1) / N).astype(np.float32).astype(np.float64)
    wts[250:350] = 0.0
    x, h = _pair(orc, 41, M, N)
    nu = np.zeros(1)
    ctx = api.Context(M, N, 4, nu, k_lo, k_hi, weights=wts, eps=0.5, r_n=10)
    gx = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h), grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    r = orc.loss(x, h, nu, k_lo, k_hi, weights=wts, eps=0.5)
    assert abs(t[1] - r["wpsl"]) <= CHI_TOL
    cell = int(t[6 + int(t[5])])
    assert not (250 <= cell % D < 350)
    _, ogx, ogh = orc.grad_xh(x, h, nu, k_lo, k_hi, weights=wts, eps=0.5, use_cell=cell)
    scale = max(np.max(np.abs(ogx)), np.max(np.abs(ogh)))
    assert np.max(np.abs(gx.cpu().numpy() - ogx)) <= 1e-4 * scale
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 1e-4 * scale
    ctx.close()


def test_corr_fp64_acceptance(api, orc):
    w = wl.correlation()
    b = wl.phase_indices(3, w.M, w.N, w.B)
    u = orc.init_logits(b, w.B, 10).astype(np.float32)
    _, h = _pair(orc, 3, w.M, w.N, 0.2)
    ctx = api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, r_n=10)
    out = ctx.af_eval_hard(_dev(u), _dev(h))
    x = np.exp(2j * np.pi * b / w.B)
    met, snrl = orc.metrics(x, h, w.nu, w.k_lo, w.k_hi)
    np.testing.assert_allclose(out[:4], met, atol=1e-8)
    np.testing.assert_allclose(out[4:], snrl, atol=1e-8)
    ctx.close()


def test_corr_optimiser_improves_the_correlation_design(api, orc):
    """SQNGD on the correlation setting for 50 outer iterations: finite log,
    the FP64 PSLR of the hard design improves on the random start."""
    w = wl.correlation()
    b = torch.from_numpy(wl.phase_indices(4, w.M, w.N, w.B)).cuda()
    ctx = api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db, r_n=w.r_n, c=w.c,
                      lr_h=w.lr_h, lr_x=w.lr_x)
    u, h = ctx.sqngd_init(b)
    start = ctx.af_eval_hard(u, h)
    st = api.SqngdState.create(u, h)
    log = ctx.sqngd_step(st, 50)
    assert np.isfinite(log).all()
    end = ctx.af_eval_hard(st.u, st.h)
    assert end[2] < start[2] - 1.0, (start[2], end[2])
    ctx.close()
