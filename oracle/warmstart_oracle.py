"""FP64 CPU oracle of the learned warm-start network (NumPy).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and
``bench.py``'s baseline legs are the only callers; the product package never
imports this module and this module imports nothing from it.

The paper generates the continuous transmit phases with a network f_theta
whose input is the initial phase configuration y0 (Section II-B, Eq. 17;
Section IV describes a ResNet; its oracle is oracle/resnet_oracle.py).  The
default transmit parameters are direct logits u optimised by SQNGD, with a
small convolutional warm-start network, not in the paper, proposing the
initial code.
What this file computes is therefore its own plain definition:

  features F[c][n] (n = 0..N-1, 32 channels):
      c = 0             n / N
      c = 1 + 2i, 2+2i  cos, sin of 2 pi f_i n / N, f_i = 1, 2, 4, 8
      c = 9 .. 13       the five conditioning scalars cond[0..4], broadcast
      c = 14 + 2m, 15+2m  cos, sin of 2 pi b0[m][n] / B for waveform m < M
                        (the random initial code, the "seed" channel; 0 for m >= M)
      c = 22 .. 31      0
  layer l = 1..4:  z_l[co][n] = bias_l[co] + sum_ci sum_t W_l[co][ci][t] h_{l-1}[ci][n + t - 2]
                   (h outside [0, N) is 0), h_l = tanh(z_l) for l < 4, logits = z_4
  logits channel m * 16 + q is the score of phase level q for waveform m (q < B).
  loss (one design) = mean over m < M, n < N of  -log softmax_{q < B}(logits[m*16+q][n])[target[m][n]]
  loss (batch) = mean over designs.
  weights W_l are FP16 values (biases FP32); Adam (0.9, 0.999, 1e-8, bias
  corrected) updates FP32 master copies and the FP16 weights are their
  round-to-nearest-even images.

parity unpinned by the paper (not in the paper); pinned instead by a
brute-force convolution, central finite differences of the loss, the
cross-entropy closed forms, translation equivariance and torch's Adam.
"""
from __future__ import annotations

import numpy as np

CIN = 32          # input feature channels
CH = 64           # hidden and output channels
KW = 5            # kernel width
PAD = 2
QMAX = 16         # phase levels per waveform in the output channels
MMAX = 4          # waveforms in the output channels
FREQS = (1, 2, 4, 8)


def layer_shapes(cin: int = CIN, ch: int = CH, kw: int = KW, layers: int = 4):
    """[(cout, cin, kw)] of the four convolutions."""
    return [(ch, cin, kw)] + [(ch, ch, kw)] * (layers - 1)


def init_params(seed: int, cin: int = CIN, ch: int = CH, kw: int = KW, layers: int = 4):
    """Seeded starting point: W ~ N(0, 1/(cin*kw)) rounded to FP16, biases 0."""
    rng = np.random.default_rng(seed)
    params = []
    for co, ci, k in layer_shapes(cin, ch, kw, layers):
        w = rng.standard_normal((co, ci, k)) / np.sqrt(ci * k)
        params.append({"W": to_fp16(w), "b": np.zeros(co)})
    return params


def to_fp16(w):
    """Round to the nearest FP16 value (ties to even), returned as float64."""
    return np.asarray(w, dtype=np.float64).astype(np.float16).astype(np.float64)


def features(b0, M: int, N: int, B: int, cond, cin: int = CIN):
    """Input features of one design (see the module docstring). b0: [M, N] ints."""
    F = np.zeros((cin, N))
    n = np.arange(N, dtype=np.float64)
    F[0] = n / N
    for i, f in enumerate(FREQS):
        F[1 + 2 * i] = np.cos(2 * np.pi * f * n / N)
        F[2 + 2 * i] = np.sin(2 * np.pi * f * n / N)
    for i in range(5):
        F[9 + i] = cond[i]
    for m in range(M):
        ph = 2 * np.pi * np.asarray(b0[m], dtype=np.float64) / B
        F[14 + 2 * m] = np.cos(ph)
        F[15 + 2 * m] = np.sin(ph)
    return F


def conv(W, bias, h):
    """z[co][n] = bias[co] + sum_ci sum_t W[co][ci][t] h[ci][n + t - pad] (zero padding)."""
    co, ci, kw = W.shape
    pad = (kw - 1) // 2
    N = h.shape[1]
    hp = np.zeros((ci, N + 2 * pad))
    hp[:, pad:pad + N] = h
    z = np.tile(bias[:, None], (1, N)).astype(np.float64)
    for t in range(kw):
        z += W[:, :, t] @ hp[:, t:t + N]
    return z


def forward(params, F):
    """Activations of every layer: hs[0] = F, hs[l] = tanh(z_l), last entry = logits."""
    hs = [F]
    for li, p in enumerate(params):
        z = conv(p["W"], p["b"], hs[-1])
        hs.append(z if li == len(params) - 1 else np.tanh(z))
    return hs


def design_loss_grad_logits(logits, target, M: int, B: int):
    """Cross-entropy of one design and its gradient with respect to the logits."""
    N = logits.shape[1]
    g = np.zeros_like(logits)
    loss = 0.0
    for m in range(M):
        s = logits[m * QMAX:m * QMAX + B]                  # [B, N]
        smax = s.max(axis=0)
        e = np.exp(s - smax)
        Z = e.sum(axis=0)
        p = e / Z
        t = np.asarray(target[m])
        loss += np.sum(np.log(Z) + smax - s[t, np.arange(N)])
        p[t, np.arange(N)] -= 1.0
        g[m * QMAX:m * QMAX + B] = p
    scale = 1.0 / (M * N)
    return loss * scale, g * scale


def backward(params, hs, g_logits):
    """Gradients of the loss with respect to every W and bias, given d loss / d logits."""
    grads = [None] * len(params)
    g = g_logits
    for li in range(len(params) - 1, -1, -1):
        W = params[li]["W"]
        co, ci, kw = W.shape
        pad = (kw - 1) // 2
        h = hs[li]
        N = h.shape[1]
        hp = np.zeros((ci, N + 2 * pad))
        hp[:, pad:pad + N] = h
        gW = np.zeros_like(W)
        for t in range(kw):
            gW[:, :, t] = g @ hp[:, t:t + N].T
        grads[li] = {"W": gW, "b": g.sum(axis=1)}
        if li > 0:
            # d loss / d h_{li}[ci][n] = sum_co sum_t W[co][ci][t] g[co][n - t + pad]
            gp = np.zeros((co, N + 2 * pad))
            gp[:, pad:pad + N] = g
            gh = np.zeros((ci, N))
            for t in range(kw):
                gh += W[:, :, t].T @ gp[:, 2 * pad - t:2 * pad - t + N]
            g = gh * (1.0 - hs[li] ** 2)                   # through tanh
    return grads


def loss_grad(params, batch):
    """Mean loss and gradients over a batch of (F, target, M, B) designs."""
    total = 0.0
    acc = None
    for F, target, M, B in batch:
        hs = forward(params, F)
        loss, gl = design_loss_grad_logits(hs[-1], target, M, B)
        gr = backward(params, hs, gl)
        total += loss
        if acc is None:
            acc = gr
        else:
            for a, b in zip(acc, gr):
                a["W"] += b["W"]
                a["b"] += b["b"]
    nb = len(batch)
    for a in acc:
        a["W"] /= nb
        a["b"] /= nb
    return total / nb, acc


def adam_step(master, params, grads, state, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on the FP32 master weights; params get their FP16 images.

    master / params / grads: lists of {"W", "b"}; state: {"t": int, "m": [...], "v": [...]}.
    """
    state["t"] += 1
    t = state["t"]
    if "m" not in state:
        state["m"] = [{k: np.zeros_like(v) for k, v in g.items()} for g in grads]
        state["v"] = [{k: np.zeros_like(v) for k, v in g.items()} for g in grads]
    for li, g in enumerate(grads):
        for k in ("W", "b"):
            m_ = state["m"][li][k] = b1 * state["m"][li][k] + (1 - b1) * g[k]
            v_ = state["v"][li][k] = b2 * state["v"][li][k] + (1 - b2) * g[k] ** 2
            mh = m_ / (1 - b1 ** t)
            vh = v_ / (1 - b2 ** t)
            master[li][k] = master[li][k] - lr * mh / (np.sqrt(vh) + eps)
        params[li]["W"] = to_fp16(master[li]["W"])
        params[li]["b"] = master[li]["b"].astype(np.float32).astype(np.float64)
    return master, params


def infer(params, F, M: int, B: int):
    """Phase indices b[m][n] = argmax_{q < B} logits[m*16+q][n] (lowest q on ties)."""
    logits = forward(params, F)[-1]
    return np.stack([np.argmax(logits[m * QMAX:m * QMAX + B], axis=0) for m in range(M)]).astype(np.int32)


def flatten(params):
    """All parameters in the packed order [W1, b1, W2, b2, W3, b3, W4, b4]."""
    return np.concatenate([np.concatenate([p["W"].ravel(), p["b"].ravel()]) for p in params])


def unflatten(vec, cin: int = CIN, ch: int = CH, kw: int = KW, layers: int = 4):
    out, o = [], 0
    for co, ci, k in layer_shapes(cin, ch, kw, layers):
        nw = co * ci * k
        out.append({"W": np.array(vec[o:o + nw], dtype=np.float64).reshape(co, ci, k),
                    "b": np.array(vec[o + nw:o + nw + co], dtype=np.float64)})
        o += nw + co
    return out
