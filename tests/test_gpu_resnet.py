"""Transmit-side ResNet generator (Eq. 17, Section IV architecture) on the GPU
against the FP64 oracle (oracle/resnet_oracle.py), through the C ABI: the
forward pass, one Adam step from a given dL/du, one SQNGD outer iteration with
the generator attached, and a short run compared statistically."""
import numpy as np
import pytest
import torch

import oracle.resnet_oracle as rno
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


def _theta(P, seed, z0=None):
    """Oracle initialisation with a non-zero output layer (every path active)."""
    z0 = np.full(P, 0.4) if z0 is None else z0
    th = rno.init_params(P, z0, lambda n: wl.uniform(seed, n, 3))
    parts = rno.unflatten(th, P)
    parts[-2] = (wl.uniform(seed, parts[-2].size, 4).reshape(parts[-2].shape) - 0.5) * 0.2
    for i in range(1, len(parts) - 2, 2):
        parts[i] = (wl.uniform(seed + i, parts[i].size, 5) - 0.5) * 0.2
    return rno.flatten(parts).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("P", [2048, 100, 7])
def test_forward_matches_oracle(api, P):
    th = _theta(P, 1)
    y0 = wl.uniform(2, P, 1).astype(np.float32)
    rn = api.ResNetGenerator(P)
    rn.set_params(th)
    u = rn.forward(_dev(y0)).cpu().numpy()
    ref, _ = rno.forward(th, y0.astype(np.float64))
    assert np.max(np.abs(u - ref)) <= 2e-5 * max(1.0, np.max(np.abs(ref)))
    np.testing.assert_array_equal(rn.get_params(), th.astype(np.float32))
    rn.close()


@pytest.mark.parametrize("P", [2048, 100])
def test_train_step_matches_oracle(api, P):
    lr = 1e-3
    th = _theta(P, 3)
    y0 = wl.uniform(4, P, 1).astype(np.float32)
    du = wl.normal(5, P, 1).astype(np.float32)
    rn = api.ResNetGenerator(P)
    rn.set_params(th)
    rn.forward(_dev(y0))
    u1 = rn.train_step(_dev(y0), _dev(du), lr, 1).cpu().numpy()
    got = rn.get_params().astype(np.float64)
    _, cache = rno.forward(th, y0.astype(np.float64))
    g = rno.backward(th, cache, du.astype(np.float64))
    exp = th.copy()
    rno.adam(exp, g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    # Adam's first step moves each parameter by about lr sign(g); FP32 and FP64
    # gradients differ only where |g| is near Adam's eps
    d = np.abs(got - exp)
    assert np.max(d) <= 0.05 * lr + 2e-6, np.max(d)
    assert np.mean(d <= 1e-3 * lr + 2e-6) > 0.999
    ref_u, _ = rno.forward(exp, y0.astype(np.float64))
    assert np.max(np.abs(u1 - ref_u)) <= 1e-4 * max(1.0, np.max(np.abs(ref_u)))
    rn.close()


def _start(orc, w, seed):
    b = wl.phase_indices(seed, w.M, w.N, w.B)
    z0 = ((w.r_n // 2) * w.B + b.astype(np.float64)) / (w.B * w.r_n)
    y0 = (b.astype(np.float64) / w.B).ravel()            # Y0 = Y / (2 pi), the normalised phases
    h0 = orc.project(np.exp(2j * np.pi * b / w.B)).astype(np.complex64)
    return b, z0, y0, h0


def test_outer_iteration_with_generator(api, orc):
    """n_h = 0, n_x = 1: the finish kernel's dL/du drives one Adam step of the
    generator; parameters and u afterwards against the oracle step from the
    same dL/du (af_loss_grad at the start)."""
    w = wl.small(2, 64, 4, 64, r_n=10)
    lr = 1e-3
    b, z0, y0, h0 = _start(orc, w, 7)
    P = w.M * w.N
    th = rno.init_params(P, z0.ravel(), lambda n: wl.uniform(8, n, 3)).astype(np.float32).astype(np.float64)
    rn = api.ResNetGenerator(P)
    rn.set_params(th)
    ctx = api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, r_n=w.r_n, n_h=0, n_x=1, lr_x=lr)
    y0d = _dev(y0.astype(np.float32))
    u0 = rn.forward(y0d).reshape(w.M, w.N)
    np.testing.assert_allclose(torch.sigmoid(u0).cpu().numpy(), z0, atol=1e-6)   # the network starts at z0
    gu = torch.empty((w.M, w.N), dtype=torch.float32, device="cuda")
    ctx.af_loss_grad(u0.contiguous(), _dev(h0), use_hard=False, grad_u=gu)
    du = gu.cpu().numpy().ravel().astype(np.float64)
    ctx.attach_generator(rn, y0d)
    st = api.SqngdState.create(u0.contiguous(), _dev(h0))
    log = ctx.sqngd_step(st, 1)
    assert np.isfinite(log).all()
    got = rn.get_params().astype(np.float64)
    _, cache = rno.forward(th, y0)
    g = rno.backward(th, cache, du)
    exp = th.copy()
    rno.adam(exp, g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    d = np.abs(got - exp)
    assert np.max(d) <= 0.05 * lr + 2e-6 and np.mean(d <= 1e-3 * lr + 2e-6) > 0.999
    ref_u, _ = rno.forward(exp, y0)
    assert np.max(np.abs(st.u.cpu().numpy().ravel() - ref_u)) <= 1e-4 * max(1.0, np.max(np.abs(ref_u)))
    ctx.close()
    rn.close()


def test_generator_run_improves_and_tracks_oracle(api, orc):
    """60 outer iterations of the tiny problem with the generator (r_n = 10,
    lr 1e-3) from 3 seeds: the hard PSLR improves on the start on both sides
    and the medians agree within 0.5 dB."""
    w = wl.tiny()
    r_n, lr, n_outer = 10, 1e-3, 60
    rho, a = orc.thresholds(w.B, r_n)
    rho32 = rho.astype(np.float32).astype(np.float64)
    g_final, o_final = [], []
    for seed in range(3):
        b, z0, y0, h0 = _start(orc, wl.small(w.M, w.N, w.B, w.L, w.k_lo, w.k_hi, r_n=r_n), seed)
        P = w.M * w.N
        th = rno.init_params(P, z0.ravel(), lambda n: wl.uniform(20 + seed, n, 3)).astype(np.float32).astype(np.float64)
        rn = api.ResNetGenerator(P)
        rn.set_params(th)
        ctx = api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db, r_n=r_n, c=w.c,
                          lr_h=w.lr_h, lr_x=lr)
        y0d = _dev(y0.astype(np.float32))
        u0 = rn.forward(y0d).reshape(w.M, w.N).contiguous()
        ctx.attach_generator(rn, y0d)
        st = api.SqngdState.create(u0, _dev(h0))
        start = ctx.af_eval_hard(st.u, st.h)
        log = ctx.sqngd_step(st, n_outer)
        assert np.isfinite(log).all()
        out = ctx.af_eval_hard(st.u, st.h)
        assert out[2] < start[2]
        g_final.append(out[2])
        ctx.close()
        rn.close()
        # oracle: the same loop with the network in FP64
        thv, m, v = th.copy(), np.zeros_like(th), np.zeros_like(th)
        h = h0.astype(np.complex128)
        mh, vh = np.zeros_like(h), np.zeros_like(h)
        t_x = t_h = 0
        u, cache = rno.forward(thv, y0)
        for _ in range(n_outer):
            _, xh = orc.hard_waveform(u.reshape(w.M, w.N), rho32, w.B)
            for _i in range(w.n_h):
                _, _, gh = orc.grad_xh(xh, h, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db)
                t_h += 1
                hv = h.view(np.float64).ravel().copy()
                mhv, vhv = mh.view(np.float64).ravel().copy(), vh.view(np.float64).ravel().copy()
                orc.adam(hv, gh.view(np.float64).ravel(), mhv, vhv, t_h, w.lr_h)
                h = orc.project(hv.view(np.complex128).reshape(w.M, w.N))
                mh, vh = mhv.view(np.complex128).reshape(w.M, w.N), vhv.view(np.complex128).reshape(w.M, w.N)
            for _j in range(w.n_x):
                _, gu, _ = orc.loss_grad_u(u.reshape(w.M, w.N), h, rho32, a, w.c, w.nu, w.k_lo, w.k_hi,
                                           eps=w.eps, snrl_db=w.snrl_db)
                t_x += 1
                g = rno.backward(thv, cache, gu.ravel())
                rno.adam(thv, g, m, v, t_x, lr)
                u, cache = rno.forward(thv, y0)
        _, xo = orc.hard_waveform(u.reshape(w.M, w.N), rho32, w.B)
        met, _ = orc.metrics(xo, h, w.nu, w.k_lo, w.k_hi)
        o_final.append(met[2])
    assert abs(np.median(g_final) - np.median(o_final)) <= 0.5, (g_final, o_final)
