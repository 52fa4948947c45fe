"""The allocation-free entry point af_loss_terms_noalloc against af_loss_grad_xh.

af_loss_terms_noalloc exists for callers that cannot call cudaMalloc (code
inside a stream capture, hosts whose framework owns the device memory pool,
latency-critical loops); it keeps its scratch in a fixed device array.  This
file is collected last so a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CHI_TOL = 1e-5


def _inputs(orc, seed, M, N):
    x = wl.unit_phasors(seed, M, N).astype(np.complex64)
    h = orc.project(x.astype(np.complex128) + 0.3 * wl.complex_normal(seed, M, N)).astype(np.complex64)
    return torch.from_numpy(x).cuda(), torch.from_numpy(h).cuda()


def test_noalloc_terms_match_context_path_on_two_calls(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import _lib, api
    lib = _lib.load()
    M, N, L = 3, 200, 256
    nu0, k_lo, k_hi, eps, snrl_db = -0.5, -150, 170, 0.2, 0.7
    nu = nu0 + np.arange(L) / L
    ctx = api.Context(M, N, 4, nu, k_lo, k_hi, eps=eps, snrl_db=snrl_db, r_n=10)
    stream = torch.cuda.current_stream()
    for seed in (41, 42):                       # two calls in a row share the scratch array
        x, h = _inputs(orc, seed, M, N)
        ref, _, _ = ctx.af_loss_grad_xh(x, h)
        got = torch.full((8 + M,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.af_loss_terms_noalloc(M, N, L, ctypes.c_double(nu0), k_lo, k_hi, ctypes.c_double(eps),
                                       ctypes.c_double(snrl_db), ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(got.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))
        assert st == _lib.AF_OK
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        np.testing.assert_allclose(g[:5], r[:5], rtol=0, atol=CHI_TOL)   # L, L_WPSL, WAPSL, WCPSL, L_SNRL
        np.testing.assert_array_equal(g[5:8], r[5:8])                    # class and argmax cells
        np.testing.assert_allclose(g[8:], r[8:], rtol=0, atol=1e-12)     # p_m
    ctx.close()


def test_noalloc_rejects_oversized_problems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import _lib
    lib = _lib.load()
    x = torch.zeros((1, 16), dtype=torch.complex64, device="cuda")
    t = torch.zeros(9, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p
    for M, N, L, why in ((17, 16, 32, "M must be in 1..16"), (1, 5000, 32, "N must be in 2..4096"),
                         (1, 16, 8192, "L must be a power of two"), (1, 16, 48, "L must be a power of two")):
        st = lib.af_loss_terms_noalloc(M, N, L, ctypes.c_double(-0.5), 0, 1, ctypes.c_double(0.1),
                                       ctypes.c_double(0.5), p(x.data_ptr()), p(x.data_ptr()), p(t.data_ptr()), None)
        assert st == _lib.AF_ERR_INVALID_ARG
        # the reason is readable on this thread through af_last_error(NULL)
        msg = lib.af_last_error(None).decode()
        assert msg.startswith("af_loss_terms_noalloc:") and why in msg, msg
