"""Pins of the warm-start network oracle (CPU, FP64).

The network is not in the paper, so each part is checked against something
other than itself: a brute-force convolution loop, central finite
differences of the loss, cross-entropy closed forms, translation
equivariance and PyTorch's Adam.
"""
import numpy as np
import pytest

from oracle import warmstart_oracle as wo


def _brute_conv(W, bias, h):
    co, ci, kw = W.shape
    pad = (kw - 1) // 2
    N = h.shape[1]
    z = np.zeros((co, N))
    for o in range(co):
        for n in range(N):
            acc = bias[o]
            for i in range(ci):
                for t in range(kw):
                    p = n + t - pad
                    if 0 <= p < N:
                        acc += W[o, i, t] * h[i, p]
            z[o, n] = acc
    return z


def test_conv_matches_brute_force_loop():
    rng = np.random.default_rng(1)
    for (co, ci, kw, N) in [(2, 3, 5, 7), (4, 2, 3, 1), (3, 5, 5, 2), (1, 1, 5, 9)]:
        W = rng.standard_normal((co, ci, kw))
        b = rng.standard_normal(co)
        h = rng.standard_normal((ci, N))
        np.testing.assert_allclose(wo.conv(W, b, h), _brute_conv(W, b, h), rtol=1e-13, atol=1e-13)


def test_conv_is_translation_equivariant_away_from_edges():
    rng = np.random.default_rng(2)
    W = rng.standard_normal((3, 4, 5))
    b = rng.standard_normal(3)
    h = np.zeros((4, 40))
    h[:, 10:25] = rng.standard_normal((4, 15))
    z0 = wo.conv(W, b, h)
    z1 = wo.conv(W, b, np.roll(h, 6, axis=1))
    np.testing.assert_allclose(z1[:, 14:35], z0[:, 8:29], rtol=1e-13, atol=1e-13)


def test_cross_entropy_closed_forms():
    M, B, N = 2, 5, 7
    logits = np.zeros((wo.MMAX * wo.QMAX, N))
    target = np.array([[0, 1, 2, 3, 4, 0, 1], [4, 4, 4, 4, 4, 4, 4]])
    loss, g = wo.design_loss_grad_logits(logits, target, M, B)
    assert abs(loss - np.log(B)) < 1e-14                      # uniform softmax
    for m in range(M):
        exp = np.full((B, N), 1.0 / B)
        exp[target[m], np.arange(N)] -= 1.0
        np.testing.assert_allclose(g[m * wo.QMAX:m * wo.QMAX + B], exp / (M * N), atol=1e-15)
    assert not np.any(g[M * wo.QMAX:])                        # unused channels get no gradient
    big = logits.copy()
    for m in range(M):
        big[m * wo.QMAX + target[m], np.arange(N)] = 60.0
    loss_big, _ = wo.design_loss_grad_logits(big, target, M, B)
    assert loss_big < 1e-20                                   # ~ (B-1) e^-60


def test_features_layout():
    M, N, B = 2, 8, 4
    b0 = np.array([[0, 1, 2, 3, 0, 1, 2, 3], [3, 3, 3, 3, 0, 0, 0, 0]])
    cond = [0.25, 0.5, 0.0625, 1.0, 0.05]
    F = wo.features(b0, M, N, B, cond)
    assert F.shape == (wo.CIN, N)
    np.testing.assert_allclose(F[0], np.arange(N) / N)
    np.testing.assert_allclose(F[1], np.cos(2 * np.pi * np.arange(N) / N), atol=1e-15)
    np.testing.assert_allclose(F[8], np.sin(2 * np.pi * 8 * np.arange(N) / N), atol=1e-12)
    for i in range(5):
        assert np.all(F[9 + i] == cond[i])
    np.testing.assert_allclose(F[14], [1, 0, -1, 0, 1, 0, -1, 0], atol=1e-15)      # cos(pi b / 2)
    np.testing.assert_allclose(F[17], [-1, -1, -1, -1, 0, 0, 0, 0], atol=1e-15)    # sin for waveform 1
    assert not np.any(F[18:])


def _tiny(seed):
    params = wo.init_params(seed, cin=3, ch=16, kw=3)
    rng = np.random.default_rng(seed)
    for p in params:                       # FD works on the FP64 values; no FP16 rounding here
        p["W"] = p["W"] + 0.1 * rng.standard_normal(p["W"].shape)
        p["b"] = 0.1 * rng.standard_normal(p["b"].shape)
    batch = []
    for d in range(2):
        N = 6 + d
        F = rng.standard_normal((3, N))
        target = rng.integers(0, 3, (1, N))
        batch.append((F, target, 1, 3))
    return params, batch


def test_gradient_matches_central_finite_differences():
    params, batch = _tiny(5)
    loss, grads = wo.loss_grad(params, batch)
    rng = np.random.default_rng(6)
    h = 1e-6
    for li in range(len(params)):
        for key in ("W", "b"):
            arr = params[li][key]
            for _ in range(6):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = wo.loss_grad(params, batch)
                arr[idx] = old - h
                lm, _ = wo.loss_grad(params, batch)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - grads[li][key][idx]) <= 1e-7 * max(1.0, abs(fd)), (li, key, idx)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    master = [{"W": rng.standard_normal((2, 3, 5)), "b": rng.standard_normal(2)}]
    params = [{"W": wo.to_fp16(master[0]["W"]), "b": master[0]["b"].copy()}]
    tw = torch.tensor(master[0]["W"], dtype=torch.float64, requires_grad=True)
    tb = torch.tensor(master[0]["b"], dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tw, tb], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    state = {"t": 0}
    for step in range(4):
        gw = rng.standard_normal((2, 3, 5))
        gb = rng.standard_normal(2)
        wo.adam_step(master, params, [{"W": gw, "b": gb}], state, 1e-2)
        tw.grad = torch.tensor(gw)
        tb.grad = torch.tensor(gb)
        opt.step()
        np.testing.assert_allclose(master[0]["W"], tw.detach().numpy(), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(master[0]["b"], tb.detach().numpy(), rtol=1e-12, atol=1e-14)
    # the forward weights are the FP16 images of the master copies
    torch16 = torch.tensor(master[0]["W"]).to(torch.float16).to(torch.float64).numpy()
    np.testing.assert_array_equal(params[0]["W"], torch16)


def test_flatten_round_trip_and_parameter_count():
    params = wo.init_params(3)
    vec = wo.flatten(params)
    assert vec.size == 64 * 32 * 5 + 3 * 64 * 64 * 5 + 4 * 64
    back = wo.unflatten(vec)
    for a, b in zip(params, back):
        np.testing.assert_array_equal(a["W"], b["W"])
        np.testing.assert_array_equal(a["b"], b["b"])


def test_infer_takes_lowest_level_on_ties():
    params = wo.init_params(4)
    for p in params:
        p["W"][:] = 0.0
    params[-1]["b"][:] = 0.0
    params[-1]["b"][3] = 1.0                 # waveform 0 prefers level 3
    params[-1]["b"][wo.QMAX + 1] = 1.0       # waveform 1 prefers level 1
    F = wo.features(np.zeros((2, 10), int), 2, 10, 4, [0.0] * 5)
    b = wo.infer(params, F, 2, 4)
    assert np.all(b[0] == 3) and np.all(b[1] == 1)
    params[-1]["b"][:] = 0.0
    assert np.all(wo.infer(params, F, 2, 4) == 0)            # all tied -> level 0
