"""FP64 oracle of the transmit-side ResNet generator z = f_theta(y0) (Section
III-A, Eq. 17; architecture of Section IV: 5 residual blocks, hidden width
128, tanh in the hidden and residual layers, sigmoid at the output).

TEST INFRASTRUCTURE ONLY: the test suite and the smoke check are the only
callers; the product package never imports this module.

Architecture (READING: the paper names the block count, the width and the
activations; the block wiring is the standard two-layer residual block):
    a   = W_in y0 + b_in,          h_0 = tanh(a)                 W_in: [H][P]
    q_k = W1_k h_{k-1} + b1_k,     r_k = tanh(q_k)               W1_k: [H][H]
    s_k = h_{k-1} + W2_k r_k + b2_k, h_k = tanh(s_k)   k = 1..5  W2_k: [H][H]
    u   = W_out h_5 + b_out,       z = sigmoid(u)                W_out: [P][H]
with P = N M the number of phases (y0 = vec(Y0) of Eq. 16).  u is the
pre-sigmoid output; the loss reaches it through dL/du, the same quantity the
direct-logit form of the transmit chain differentiates.

Parameters are kept in one flat vector in the order
    W_in, b_in, (W1_k, b1_k, W2_k, b2_k) for k = 1..5, W_out, b_out
with every matrix row-major.
"""
from __future__ import annotations

import numpy as np

BLOCKS = 5
WIDTH = 128


def shapes(P: int, H: int = WIDTH, blocks: int = BLOCKS):
    s = [(H, P), (H,)]
    for _ in range(blocks):
        s += [(H, H), (H,), (H, H), (H,)]
    s += [(P, H), (P,)]
    return s


def param_count(P: int, H: int = WIDTH, blocks: int = BLOCKS) -> int:
    return int(sum(int(np.prod(t)) for t in shapes(P, H, blocks)))


def unflatten(theta, P: int, H: int = WIDTH, blocks: int = BLOCKS):
    out, o = [], 0
    for t in shapes(P, H, blocks):
        n = int(np.prod(t))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(t))
        o += n
    assert o == len(theta)
    return out


def flatten(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def forward(theta, y0, H: int = WIDTH, blocks: int = BLOCKS):
    """Returns (u, cache) for the flat parameter vector theta and input y0 [P]."""
    y0 = np.asarray(y0, dtype=np.float64)
    P = y0.size
    p = unflatten(theta, P, H, blocks)
    W_in, b_in = p[0], p[1]
    h = np.tanh(W_in @ y0 + b_in)
    hs, rs = [h], []
    for k in range(blocks):
        W1, b1, W2, b2 = p[2 + 4 * k: 6 + 4 * k]
        r = np.tanh(W1 @ h + b1)
        h = np.tanh(h + W2 @ r + b2)
        rs.append(r)
        hs.append(h)
    W_out, b_out = p[-2], p[-1]
    u = W_out @ h + b_out
    return u, (y0, hs, rs)


def backward(theta, cache, du, H: int = WIDTH, blocks: int = BLOCKS):
    """Gradient of a loss w.r.t. theta given du = dL/du (chain rule through the
    architecture above, in reverse).  Returns the flat gradient."""
    y0, hs, rs = cache
    P = y0.size
    p = unflatten(theta, P, H, blocks)
    du = np.asarray(du, dtype=np.float64)
    g = [None] * len(p)
    W_out = p[-2]
    g[-2] = np.outer(du, hs[-1])
    g[-1] = du.copy()
    dh = W_out.T @ du
    for k in reversed(range(blocks)):
        W1, b1, W2, b2 = p[2 + 4 * k: 6 + 4 * k]
        h_prev, r, h = hs[k], rs[k], hs[k + 1]
        ds = dh * (1.0 - h * h)
        g[4 + 4 * k] = np.outer(ds, r)        # W2
        g[5 + 4 * k] = ds.copy()              # b2
        dq = (W2.T @ ds) * (1.0 - r * r)
        g[2 + 4 * k] = np.outer(dq, h_prev)   # W1
        g[3 + 4 * k] = dq.copy()              # b1
        dh = ds + W1.T @ dq
    da = dh * (1.0 - hs[0] * hs[0])
    g[0] = np.outer(da, y0)
    g[1] = da.copy()
    return flatten(g)


def adam(theta, g, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """Bias-corrected Adam, in place on float64 arrays."""
    m *= b1
    m += (1 - b1) * g
    v *= b2
    v += (1 - b2) * g * g
    theta -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)


def init_params(P: int, z0, seed_uniform, H: int = WIDTH, blocks: int = BLOCKS):
    """READING of the initialisation, which Algorithm 1 leaves open: the hidden
    layers draw U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from the caller's uniform [0,1)
    stream and zero biases; the output layer starts at W_out = 0 and
    b_out = logit(z0), so that z = z0 at the start -- the same initial design
    as the direct-logit form.  seed_uniform(count) -> uniform draws."""
    parts = []
    for i, t in enumerate(shapes(P, H, blocks)):
        n = int(np.prod(t))
        if i == len(shapes(P, H, blocks)) - 2:
            parts.append(np.zeros(n))
        elif i == len(shapes(P, H, blocks)) - 1:
            z = np.asarray(z0, dtype=np.float64).ravel()
            parts.append(np.log(z / (1.0 - z)))
        elif len(t) == 1:
            parts.append(np.zeros(n))
        else:
            bound = 1.0 / np.sqrt(t[1])
            parts.append((2.0 * seed_uniform(n) - 1.0) * bound)
    return flatten(parts)
