"""The largest sizes the ABI accepts, against the FP64 oracle: M = 16
waveforms, N = 4096 chips (folded into a short transform), B = 1024 levels,
and K = 8192 trained thresholds."""
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


@pytest.mark.parametrize("M,N,L,k_lo,k_hi", [(16, 64, 64, -63, 63), (1, 4096, 32, -40, 40), (2, 4096, 64, -3, 3)])
def test_largest_shapes_loss_and_gradient(api, orc, M, N, L, k_lo, k_hi):
    nu = wl.full_grid(L)
    x = wl.unit_phasors(90 + M, M, N).astype(np.complex64)
    h = orc.project(x.astype(np.complex128) + 0.3 * wl.complex_normal(90 + M, M, N)).astype(np.complex64)
    ctx = api.Context(M, N, 4, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5, r_n=10)
    assert ctx.path in (api.AF_PATH_FFT, api.AF_PATH_DFT)
    gx = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(_dev(x), _dev(h), grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    r = orc.loss(x, h, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5)
    for gi, key in ((2, "wapsl"), (3, "wcpsl")):
        assert abs(t[gi] - r[key]) <= 1e-5, (key, t[gi], r[key])
    np.testing.assert_allclose(t[8:8 + M], r["p"], atol=1e-6)
    cell = int(t[6 + int(t[5])])
    _, ogx, ogh = orc.grad_xh(x, h, nu, k_lo, k_hi, eps=0.3, snrl_db=0.5, use_cell=cell)
    scale = max(np.max(np.abs(ogx)), np.max(np.abs(ogh)))
    assert np.max(np.abs(gx.cpu().numpy() - ogx)) <= 1e-4 * scale
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 1e-4 * scale
    ctx.close()


def test_largest_alphabet_quantizer_bit_exact(api, orc):
    B, r_n = 1024, 1
    ctx = api.Context(2, 32, B, wl.full_grid(32), -31, 31, r_n=r_n)
    z = wl.uniform(95, 20000, 1).astype(np.float32)
    q, _ = ctx.quantize(_dev(z))
    rho, _ = orc.thresholds(B, r_n)
    oq, _ = orc.hard_quantize(z.astype(np.float64), rho.astype(np.float32).astype(np.float64), B)
    np.testing.assert_array_equal(q.cpu().numpy(), oq)
    ctx.close()


def test_largest_trained_threshold_set(api, orc):
    """K = 8192 (B = 64, r_n = 128): the gradient w.r.t. every threshold and the
    projection, against the oracle."""
    M, N, L, B, r_n, c = 2, 64, 64, 64, 128, 300.0
    nu = wl.full_grid(L)
    u = wl.logits(96, M, N, 1.5).astype(np.float32)
    h = orc.project(wl.unit_phasors(96, M, N) + 0.2 * wl.complex_normal(96, M, N)).astype(np.complex64)
    ctx = api.Context(M, N, B, nu, -(N - 1), N - 1, eps=0.25, r_n=r_n, c=c, n_h=0, n_x=1, train_rho=True)
    terms, _, _, gr = ctx.af_loss_grad_rho(_dev(u), _dev(h))
    ctx.af_sync()
    t = terms.cpu().numpy()
    rho, a = orc.thresholds(B, r_n)
    rho = rho.astype(np.float32).astype(np.float64)
    cell = int(t[6 + int(t[5])])
    _, _, ogr = orc.loss_grad_u_rho(u.astype(np.float64), h, rho, a, c, nu, -(N - 1), N - 1, eps=0.25,
                                    use_cell=cell)
    g = gr.cpu().numpy()
    assert g.size == 8192
    assert np.max(np.abs(g - ogr)) <= 2e-3 * np.max(np.abs(ogr))
    r = (rho + (wl.uniform(97, rho.size, 1) - 0.5) * 4e-4).astype(np.float32)
    got = ctx.af_project_thresholds(_dev(r)).cpu().numpy()
    np.testing.assert_allclose(got, orc.project_thresholds(r.astype(np.float64)), atol=2e-6)
    ctx.close()
