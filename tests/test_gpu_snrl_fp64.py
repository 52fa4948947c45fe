"""The SNRL ratio in FP64 on every forward path: p_m (Eq. 38) and L_SNRL
(Eq. 41) against the FP64 oracle to 1e-12 (absolute; p_m <= 1 for
unimodular waveforms and energy-N filters).  A_mm(0,0) is summed from exact
FP32 products in double-float (about 44 bits), then p_m and L_SNRL are
formed in FP64, so the only error left is that summation's, far below the
FP32 rounding of the inputs that both sides share."""
import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

P_TOL = 1e-12


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import api as a
    return a


CASES = [
    # M, N, nu, k_lo, k_hi, path name
    (4, 2048, wl.full_grid(2048), -2047, 2047, "AF_PATH_FFT"),
    (3, 500, wl.full_grid(256), -499, 499, "AF_PATH_FFT"),
    (4, 1024, wl.window_grid(0.1, 64), -50, 50, "AF_PATH_DFT"),
    (8, 1024, wl.window_grid(0.05, 64), -255, 255, "AF_PATH_SPLIT_BF16"),
    (2, 1200, np.zeros(1), -1199, 1199, "AF_PATH_DFT"),          # the single-bin correlation kernel
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[5]}-N{c[1]}-L{len(c[2])}")
def test_snrl_terms_are_fp64_accurate(api, orc, case):
    M, N, nu, k_lo, k_hi, path = case
    x = wl.unit_phasors(90 + N, M, N).astype(np.complex64)
    h = orc.project(x.astype(np.complex128) + 0.4 * wl.complex_normal(90 + N, M, N)).astype(np.complex64)
    ctx = api.Context(M, N, 8, nu, k_lo, k_hi, r_n=10, eps=0.1, snrl_db=0.5, path=getattr(api, path))
    terms, _, _ = ctx.af_loss_grad_xh(torch.from_numpy(x).cuda(), torch.from_numpy(h).cuda())
    ctx.af_sync()
    t = terms.cpu().numpy()
    # p_m and L_SNRL need no grid scan: Eq. 38 as numpy.vdot-style sums of the same FP32 inputs in FP64
    x64, h64 = x.astype(np.complex128), h.astype(np.complex128)
    p = np.abs(np.sum(x64 * np.conj(h64), axis=1)) / N
    ptar = 10.0 ** (-0.5 / 20.0)
    ls = np.mean((p - ptar) ** 2)
    assert np.max(np.abs(t[8:8 + M] - p)) <= P_TOL, np.max(np.abs(t[8:8 + M] - p))
    assert abs(t[4] - ls) <= P_TOL
    ctx.close()
