"""Warm-start network on the GPU (FP16 weights, FP32 accumulation) vs the FP64
oracle through the C ABI.

Tolerances: the GPU and the oracle use the same FP16 weight values; the GPU
accumulates in FP32 over at most 64*5 = 320 terms per output and computes the
features' cos/sin in FP32, so logits agree to ~1e-5 relative of their scale
(tested at 2e-4 of the largest logit); gradients to 1e-3 of the largest
gradient entry; argmax indices are compared where the oracle's top-two gap
exceeds 1e-3 (elsewhere both choices are valid).
"""
import numpy as np
import pytest
import torch

from oracle import warmstart_oracle as wo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import api as a
    return a


def _params(seed, scale=1.0):
    p = wo.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for layer in p:
        layer["W"] = wo.to_fp16(layer["W"] * scale)
        layer["b"] = (0.1 * rng.standard_normal(layer["b"].shape)).astype(np.float32).astype(np.float64)
    return p


def _batch(seed, batch, M, N, B):
    rng = np.random.default_rng(seed)
    b0 = rng.integers(0, B, (batch, M, N)).astype(np.int32)
    tg = rng.integers(0, B, (batch, M, N)).astype(np.int32)
    return b0, tg


CASES = [(2, 2, 70, 4), (3, 4, 128, 16), (1, 1, 5, 2), (4, 3, 200, 8)]   # batch, M, N, B


@pytest.mark.parametrize("case", CASES)
def test_forward_matches_oracle(api, case):
    batch, M, N, B = case
    params = _params(1)
    net = api.WarmStart(8, 256)
    net.set_params(wo.flatten(params))
    b0, _ = _batch(2, batch, M, N, B)
    cond = api.ws_cond(M, N, B, 0.05, N // 4)
    lg, b = net.forward(torch.from_numpy(b0).cuda(), B, cond)
    lg = lg.cpu().numpy()
    b = b.cpu().numpy()
    for d in range(batch):
        ref = wo.forward(params, wo.features(b0[d], M, N, B, cond))[-1]
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(lg[d] - ref)) <= 2e-4 * scale
        bi = wo.infer(params, wo.features(b0[d], M, N, B, cond), M, B)
        for m in range(M):
            s = np.sort(ref[m * 16:m * 16 + B], axis=0)
            clear = (s[-1] - s[-2]) > 1e-3 * scale
            assert np.array_equal(b[d, m][clear], bi[m][clear])
    net.close()


@pytest.mark.parametrize("case", CASES[:3])
def test_loss_and_gradient_match_oracle(api, case):
    batch, M, N, B = case
    params = _params(3, scale=2.0)
    net = api.WarmStart(8, 256)
    net.set_params(wo.flatten(params))
    b0, tg = _batch(4, batch, M, N, B)
    cond = api.ws_cond(M, N, B, 0.1, 50)
    loss, g = net.loss_grad(torch.from_numpy(b0).cuda(), torch.from_numpy(tg).cuda(), B, cond)
    data = [(wo.features(b0[d], M, N, B, cond), tg[d], M, B) for d in range(batch)]
    rloss, rg = wo.loss_grad(params, data)
    assert abs(loss - rloss) <= 1e-5 * max(1.0, abs(rloss))
    ref = wo.flatten(rg)
    assert np.max(np.abs(g - ref)) <= 1e-3 * np.max(np.abs(ref))
    net.close()


def test_adam_steps_match_oracle(api):
    batch, M, N, B = 2, 2, 64, 4
    params = _params(5)
    master = [{"W": p["W"].copy(), "b": p["b"].copy()} for p in params]
    net = api.WarmStart(4, 64)
    net.set_params(wo.flatten(params))
    b0, tg = _batch(6, batch, M, N, B)
    cond = api.ws_cond(M, N, B, 0.05, 20)
    data = [(wo.features(b0[d], M, N, B, cond), tg[d], M, B) for d in range(batch)]
    state = {"t": 0}
    d0, t0 = torch.from_numpy(b0).cuda(), torch.from_numpy(tg).cuda()
    for step in range(3):
        loss = net.train_step(d0, t0, B, cond, lr=1e-3)
        rloss, rg = wo.loss_grad(params, data)
        assert abs(loss - rloss) <= 1e-5 * max(1.0, rloss)
        wo.adam_step(master, params, rg, state, 1e-3)
    got = net.get_params()
    ref = wo.flatten(master)
    # Adam normalises each coordinate, so FP32-vs-FP64 gradient noise on tiny
    # gradient entries moves a parameter by up to ~lr per step
    assert np.max(np.abs(got - ref)) <= 3 * 1e-3 + 1e-6
    assert np.median(np.abs(got - ref)) <= 1e-5
    net.close()


def test_training_reduces_the_loss(api):
    batch, M, N, B = 8, 2, 64, 4
    net = api.WarmStart(batch, N)
    net.set_params(wo.flatten(wo.init_params(7)))
    b0, _ = _batch(8, batch, M, N, B)
    tg = (b0 + 1) % B                        # a learnable map of the input code
    cond = api.ws_cond(M, N, B, 0.05, 20)
    d0, t0 = torch.from_numpy(b0).cuda(), torch.from_numpy(tg).cuda()
    first = net.train_step(d0, t0, B, cond, lr=3e-3)
    for _ in range(150):
        last = net.train_step(d0, t0, B, cond, lr=3e-3, sync=False)
    last = net.train_step(d0, t0, B, cond, lr=3e-3)
    assert last < 0.2 * first
    _, b = net.forward(d0, B, cond, logits=False)
    assert np.mean(b.cpu().numpy() == tg) > 0.95
    net.close()


def test_bad_configurations_are_rejected(api):
    net = api.WarmStart(2, 32)
    b0 = torch.zeros((1, 5, 32), dtype=torch.int32, device="cuda")
    with pytest.raises(api.AfError, match="AF_ERR_INVALID_ARG"):
        net.forward(b0, 4, [0.0] * 5)                       # M = 5
    b0 = torch.zeros((3, 2, 32), dtype=torch.int32, device="cuda")
    with pytest.raises(api.AfError, match="AF_ERR_INVALID_ARG"):
        net.forward(b0, 4, [0.0] * 5)                       # batch > batch_max
    b0 = torch.zeros((1, 2, 33), dtype=torch.int32, device="cuda")
    with pytest.raises(api.AfError, match="AF_ERR_INVALID_ARG"):
        net.forward(b0, 4, [0.0] * 5)                       # N > n_max
    b0 = torch.zeros((1, 2, 32), dtype=torch.int32, device="cuda")
    with pytest.raises(api.AfError, match="AF_ERR_INVALID_ARG"):
        net.forward(b0, 17, [0.0] * 5)                      # B > 16
    net.close()


def test_pipeline_generates_trains_and_proposes(api):
    """The training pipeline end to end at toy sizes: converged designs from
    the optimiser, a few epochs, proposals of the right shape and range."""
    from paper_2604_25728_gb300 import warmstart as ws
    from paper_2604_25728_gb300 import workloads as wl
    data = []
    ctx = ws._ctx(2, 128, 16, 0.1, 32, 20, api.AF_PATH_SPLIT_BF16)
    for i in range(4):
        b0 = wl.phase_indices(500 + i, 2, 128, 16)
        bs = ws.converge(ctx, b0, 10)
        assert bs.shape == (2, 128) and bs.min() >= 0 and bs.max() < 16
        data.append((2, 128, b0, bs))
    ctx.close()
    net, hist = ws.train(data, epochs=3, batch=4)
    assert len(hist) == 3 and all(np.isfinite(hist)) and hist[-1] < hist[0]
    bp = ws.propose(net, data[0][2], 16, 0.1, 20)
    assert bp.shape == (2, 128) and bp.min() >= 0 and bp.max() < 16
    net.close()


def test_saved_parameters_load(api):
    from paper_2604_25728_gb300 import warmstart as ws
    params, rec = ws.load()
    assert params.size == api.WarmStart.param_count() and np.all(np.isfinite(params))
    assert rec["designs"] >= 256 and rec["held_out_index_agreement"] > 0.5
