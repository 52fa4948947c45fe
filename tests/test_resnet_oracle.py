"""Pins for the ResNet generator oracle (Eq. 17, Section IV architecture):
finite differences of a scalar loss through the whole network, the initial
output, the residual identity and Adam against torch.optim.Adam.  CPU only."""
import numpy as np
import pytest

import oracle.resnet_oracle as rn
from paper_2604_25728_gb300 import workloads as wl


def _theta(P, H, seed, out_scale=0.3):
    u = lambda n, s=[0]: (s.__setitem__(0, s[0] + 1), wl.uniform(seed * 100 + s[0], n, 5))[1]
    th = rn.init_params(P, np.full(P, 0.4), u, H=H)
    # give the output layer non-zero weights so every gradient path is exercised
    parts = rn.unflatten(th, P, H)
    parts[-2] = (wl.uniform(seed, parts[-2].size, 6).reshape(parts[-2].shape) - 0.5) * out_scale
    for i in range(1, len(parts) - 2, 2):
        parts[i] = (wl.uniform(seed + i, parts[i].size, 7) - 0.5) * 0.2
    return rn.flatten(parts)


def test_gradient_matches_finite_differences():
    """L = sum_e c_e u_e + 0.5 sum_e u_e^2 (any smooth function of u) and its
    gradient through every layer, against central differences."""
    P, H = 7, 6
    th = _theta(P, H, 1)
    y0 = wl.uniform(2, P, 1)
    c = wl.normal(3, P, 2)
    f = lambda t: float(np.dot(c, rn.forward(t, y0, H=H)[0]) + 0.5 * np.sum(rn.forward(t, y0, H=H)[0] ** 2))
    u, cache = rn.forward(th, y0, H=H)
    g = rn.backward(th, cache, c + u, H=H)
    assert g.size == rn.param_count(P, H)
    idx = np.unique((wl.uniform(4, 60, 3) * th.size).astype(int))
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += 1e-6
        tm[i] -= 1e-6
        fd = (f(tp) - f(tm)) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
    # every parameter group reached
    parts = rn.unflatten(g, P, H)
    assert all(np.max(np.abs(q)) > 0 for q in parts)


def test_initial_output_is_z0():
    """W_out = 0, b_out = logit(z0): the network starts at the given phases."""
    P = 20
    z0 = (np.arange(P) + 0.5) / P
    th = rn.init_params(P, z0, lambda n: wl.uniform(9, n, 1))
    u, _ = rn.forward(th, wl.uniform(8, P, 1))
    np.testing.assert_allclose(1 / (1 + np.exp(-u)), z0, rtol=1e-14)
    assert rn.param_count(P) == 2 * 128 * P + 128 + 5 * 2 * (128 * 128 + 128) + P


def test_zero_blocks_are_identity_through_tanh():
    """With zero block weights and biases each block maps h to tanh(h)."""
    P, H = 5, 4
    th = _theta(P, H, 3)
    parts = rn.unflatten(th, P, H)
    for i in range(2, 2 + 4 * rn.BLOCKS):
        parts[i][...] = 0.0
    th = rn.flatten(parts)
    y0 = wl.uniform(5, P, 1)
    u, (_, hs, _) = rn.forward(th, y0, H=H)
    h = np.tanh(parts[0] @ y0 + parts[1])
    for _ in range(rn.BLOCKS):
        h = np.tanh(h)
    np.testing.assert_allclose(hs[-1], h, rtol=1e-15)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    th = wl.normal(1, 30, 1)
    p = torch.tensor(th.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3)
    m, v = np.zeros_like(th), np.zeros_like(th)
    for t in range(1, 5):
        g = wl.normal(10 + t, 30, 1)
        rn.adam(th, g, m, v, t, 1e-3)
        opt.zero_grad()
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_package_initialisation_starts_at_z0():
    """The package's generator initialisation (paper_2604_25728_gb300.generator)
    has the documented layout and, run through the oracle, outputs z0."""
    pytest.importorskip("torch")
    from paper_2604_25728_gb300 import _lib
    try:
        _lib.load()
    except Exception:
        pytest.skip("library not built")
    from paper_2604_25728_gb300 import generator
    P = 12
    z0 = (np.arange(P) + 0.5) / P
    th = generator.init_params(P, z0, 3).astype(np.float64)
    assert th.size == rn.param_count(P)
    parts = rn.unflatten(th, P)
    assert np.all(parts[-2] == 0) and all(np.all(parts[i] == 0) for i in range(1, len(parts) - 2, 2))
    assert np.max(np.abs(parts[0])) <= 1 / np.sqrt(P) and np.max(np.abs(parts[2])) <= 1 / np.sqrt(128)
    u, _ = rn.forward(th, wl.uniform(4, P, 1))
    np.testing.assert_allclose(1 / (1 + np.exp(-u)), z0, rtol=1e-6)
