"""FP64 CPU oracle for the SQNGD hot path (ctypes wrapper around sqngd_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The product package never imports this module, and this module
imports nothing from the product package.

Conventions (same as the C file): complex arrays are numpy complex128 of shape
[M, N]; the ambiguity grid is [M, M, D, L] with pair (m, l) = (transmit m,
receive filter l), d = k - k_lo; weights are [D, L] or None (w = 1/N).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SQNGD_ORACLE_SOURCE / SQNGD_ORACLE_BUILD: a test hook that builds the oracle
# from another copy of the source (tests/test_oracle_mutations.py plants
# mistakes in such a copy and checks that the pins catch them).
_SRC = os.environ.get("SQNGD_ORACLE_SOURCE", os.path.join(_HERE, "sqngd_oracle.c"))
_BUILD = os.environ.get("SQNGD_ORACLE_BUILD", os.path.join(_HERE, "_build"))
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_longlong)


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _grid(nu, k_lo, k_hi, weights):
    nu = _f64(nu)
    w = None if weights is None else _f64(weights)
    if w is not None:
        assert w.shape == (k_hi - k_lo + 1, nu.size)
    return nu, w


# ---------------------------------------------------------------- Eq. 6
def ambiguity(x, h, nu, k_lo, k_hi):
    """Full grid chi[m, l, d, j] (Eq. 6, n counted from 0)."""
    x, h = _c128(x), _c128(h)
    M, N = x.shape
    nu = _f64(nu)
    D = k_hi - k_lo + 1
    out = np.zeros((M, M, D, nu.size), dtype=np.complex128)
    lib().or_ambiguity(M, N, nu.size, _d(nu), k_lo, k_hi, _d(x), _d(h), _d(out))
    return out


def ambiguity_cells(x, h, nu, k_lo, k_hi, cells):
    """chi at the given linear cell indices ((m*M + l)*D + d)*L + j."""
    x, h = _c128(x), _c128(h)
    M, N = x.shape
    nu = _f64(nu)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros(cells.size, dtype=np.complex128)
    lib().or_ambiguity_cells(M, N, nu.size, _d(nu), k_lo, k_hi, _d(x), _d(h),
                             int(cells.size), cells.ctypes.data_as(_lp), _d(out))
    return out


def fd_losses(x, h, nu, k_lo, k_hi, coords, weights=None, eps=0.1, snrl_db=0.5, pnorm=0.0):
    """Losses (Eq. 42) with one sample replaced, for central finite
    differences on grids too large to re-evaluate per coordinate: coords is a
    list of (target, row, col, v_plus, v_minus) with target 0 for x[row, col]
    and 1 for h[row, col]; returns (loss_plus, loss_minus) arrays.  chi is
    updated by the rank-one change of each replacement (Eq. 6 is linear in
    x_m(n) and in conj(h_l(p))); only the pairs of that row or column move."""
    x, h = _c128(x), _c128(h)
    M, N = x.shape
    nu, w = _grid(nu, k_lo, k_hi, weights)
    n = len(coords)
    tgt = np.ascontiguousarray([int(c[0]) for c in coords], dtype=np.int32)
    row = np.ascontiguousarray([int(c[1]) for c in coords], dtype=np.int32)
    col = np.ascontiguousarray([int(c[2]) for c in coords], dtype=np.int32)
    vp = _c128([complex(c[3]) for c in coords])
    vm = _c128([complex(c[4]) for c in coords])
    assert np.all((tgt == 0) | (tgt == 1)) and np.all((row >= 0) & (row < M)) and np.all((col >= 0) & (col < N))
    lp = np.zeros(n)
    lm = np.zeros(n)
    lib().or_fd_losses(M, N, nu.size, _d(nu), k_lo, k_hi, _d(w), ctypes.c_double(eps),
                       ctypes.c_double(snrl_db), ctypes.c_double(pnorm), _d(x), _d(h), n,
                       tgt.ctypes.data_as(_ip), row.ctypes.data_as(_ip), col.ctypes.data_as(_ip),
                       _d(vp), _d(vm), _d(lp), _d(lm))
    return lp, lm


# ---------------------------------------------------------------- loss, Eqs. 7-9, 37-42
def loss(x, h, nu, k_lo, k_hi, weights=None, eps=0.1, snrl_db=0.5, pnorm=0.0):
    """Returns dict(loss, wpsl, wapsl, wcpsl, snrl_term, cls, p[M], cells[2])."""
    x, h = _c128(x), _c128(h)
    M, N = x.shape
    nu, w = _grid(nu, k_lo, k_hi, weights)
    terms = np.zeros(6)
    p = np.zeros(M)
    cells = np.zeros(2, dtype=np.int64)
    lib().or_loss(M, N, nu.size, _d(nu), k_lo, k_hi, _d(w), ctypes.c_double(eps),
                  ctypes.c_double(snrl_db), ctypes.c_double(pnorm), _d(x), _d(h),
                  _d(terms), _d(p), cells.ctypes.data_as(_lp))
    return dict(loss=terms[0], wpsl=terms[1], wapsl=terms[2], wcpsl=terms[3],
                snrl_term=terms[4], cls=int(terms[5]), p=p, cells=cells)


def grad_xh(x, h, nu, k_lo, k_hi, weights=None, eps=0.1, snrl_db=0.5, pnorm=0.0,
            use_cell=None):
    """Analytic gradient (dL/dRe + j dL/dIm) w.r.t. x and h; returns (terms, gx, gh)."""
    x, h = _c128(x), _c128(h)
    M, N = x.shape
    nu, w = _grid(nu, k_lo, k_hi, weights)
    terms = np.zeros(6)
    gx = np.zeros_like(x)
    gh = np.zeros_like(h)
    uc = None
    if use_cell is not None:
        uc = (ctypes.c_longlong * 1)(int(use_cell))
    lib().or_grad_xh(M, N, nu.size, _d(nu), k_lo, k_hi, _d(w), ctypes.c_double(eps),
                     ctypes.c_double(snrl_db), ctypes.c_double(pnorm), _d(x), _d(h),
                     uc, _d(terms), _d(gx), _d(gh))
    return terms, gx, gh


# ---------------------------------------------------------------- quantizers, Eqs. 24, 25, 43
def thresholds(B, r_n):
    K = B * r_n
    rho = np.zeros(K)
    a = ctypes.c_double(0)
    lib().or_thresholds(B, r_n, _d(rho), ctypes.byref(a))
    return rho, a.value


def soft_quantize(z, rho, a, c):
    z = _f64(z).ravel()
    rho = _f64(rho)
    y = np.zeros_like(z)
    dy = np.zeros_like(z)
    lib().or_soft_quantize(z.size, _d(z), rho.size, _d(rho), ctypes.c_double(a),
                           ctypes.c_double(c), _d(y), _d(dy))
    return y, dy


def hard_quantize(z, rho, B):
    z = _f64(z).ravel()
    rho = _f64(rho)
    q = np.zeros(z.size, dtype=np.int32)
    b = np.zeros(z.size, dtype=np.int32)
    lib().or_hard_quantize(z.size, _d(z), rho.size, _d(rho), B,
                           q.ctypes.data_as(_ip), b.ctypes.data_as(_ip))
    return q, b


def hard_quantize_literal(z, rho, a, c):
    z = _f64(z).ravel()
    rho = _f64(rho)
    y = np.zeros_like(z)
    lib().or_hard_quantize_literal(z.size, _d(z), rho.size, _d(rho), ctypes.c_double(a),
                                   ctypes.c_double(c), _d(y))
    return y


# ---------------------------------------------------------------- projection, Adam
def project(h):
    h = _c128(h).copy()
    M, N = h.shape
    lib().or_project(M, N, _d(h))
    return h


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """In-place on float64 arrays theta, m, v."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib().or_adam(theta.size, _d(theta), _d(g), _d(m), _d(v), ctypes.c_longlong(t),
                  ctypes.c_double(lr), ctypes.c_double(b1), ctypes.c_double(b2),
                  ctypes.c_double(eps))


# ---------------------------------------------------------------- transmit chain
def soft_waveform(u, rho, a, c):
    u = _f64(u)
    M, N = u.shape
    x = np.zeros((M, N), dtype=np.complex128)
    dy = np.zeros((M, N))
    lib().or_soft_waveform(M, N, _d(u), rho.size, _d(_f64(rho)), ctypes.c_double(a),
                           ctypes.c_double(c), _d(x), _d(dy))
    return x, dy


def hard_waveform(u, rho, B):
    u = _f64(u)
    M, N = u.shape
    x = np.zeros((M, N), dtype=np.complex128)
    q = np.zeros((M, N), dtype=np.int32)
    lib().or_hard_waveform(M, N, _d(u), rho.size, _d(_f64(rho)), B, q.ctypes.data_as(_ip), _d(x))
    return q, x


def loss_grad_u(u, h, rho, a, c, nu, k_lo, k_hi, weights=None, eps=0.1, snrl_db=0.5,
                pnorm=0.0, use_cell=None):
    """Loss and gradient w.r.t. the logits u and the filters h (soft waveform)."""
    u = _f64(u)
    h = _c128(h)
    M, N = u.shape
    nu, w = _grid(nu, k_lo, k_hi, weights)
    terms = np.zeros(6)
    gu = np.zeros((M, N))
    gh = np.zeros((M, N), dtype=np.complex128)
    uc = None
    if use_cell is not None:
        uc = (ctypes.c_longlong * 1)(int(use_cell))
    lib().or_loss_grad_u(M, N, nu.size, _d(nu), k_lo, k_hi, _d(w), ctypes.c_double(eps),
                         ctypes.c_double(snrl_db), ctypes.c_double(pnorm), _d(u),
                         rho.size, _d(_f64(rho)), ctypes.c_double(a), ctypes.c_double(c),
                         _d(h), uc, _d(terms), _d(gu), _d(gh))
    return terms, gu, gh


def sqngd_outer(state, cfg):
    """One outer iteration of Algorithm 1; state is a dict of float64 arrays
    (u, h, mu, vu, mh, vh) and counters (t_x, t_h), updated in place."""
    M, N = state["u"].shape
    nu, w = _grid(cfg["nu"], cfg["k_lo"], cfg["k_hi"], cfg.get("weights"))
    rho = _f64(cfg["rho"])
    n_ev = cfg["n_h"] + cfg["n_x"]
    losses = np.zeros(n_ev)
    wpsl = np.zeros(n_ev)
    tx = ctypes.c_longlong(state["t_x"])
    th = ctypes.c_longlong(state["t_h"])
    hv = state["h"].view(np.float64)
    lib().or_sqngd_outer(
        M, N, nu.size, _d(nu), cfg["k_lo"], cfg["k_hi"], _d(w), ctypes.c_double(cfg["eps"]),
        ctypes.c_double(cfg["snrl_db"]), ctypes.c_double(cfg.get("pnorm", 0.0)),
        cfg["B"], rho.size, _d(rho), ctypes.c_double(cfg["a"]), ctypes.c_double(cfg["c"]),
        cfg["n_h"], cfg["n_x"], ctypes.c_double(cfg["lr_h"]), ctypes.c_double(cfg["lr_x"]),
        ctypes.c_double(cfg.get("b1", 0.9)), ctypes.c_double(cfg.get("b2", 0.999)),
        ctypes.c_double(cfg.get("adam_eps", 1e-8)),
        _d(state["u"]), _d(hv), _d(state["mu"]), _d(state["vu"]),
        _d(state["mh"].view(np.float64)), _d(state["vh"].view(np.float64)),
        ctypes.byref(tx), ctypes.byref(th), _d(losses), _d(wpsl))
    state["t_x"] = tx.value
    state["t_h"] = th.value
    return losses, wpsl


# ---------------------------------------------------------------- trainable thresholds
def loss_grad_u_rho(u, h, rho, a, c, nu, k_lo, k_hi, weights=None, eps=0.1, snrl_db=0.5,
                    pnorm=0.0, use_cell=None):
    """Loss of the soft waveform and its gradient w.r.t. the logits u and the
    thresholds rho (Eq. 24 with trainable rho_i); returns (terms, gu, grho)."""
    u = _f64(u)
    h = _c128(h)
    rho = _f64(rho)
    M, N = u.shape
    nu, w = _grid(nu, k_lo, k_hi, weights)
    terms = np.zeros(6)
    gu = np.zeros((M, N))
    gr = np.zeros(rho.size)
    uc = None if use_cell is None else (ctypes.c_longlong * 1)(int(use_cell))
    lib().or_loss_grad_u_rho(M, N, nu.size, _d(nu), k_lo, k_hi, _d(w), ctypes.c_double(eps),
                             ctypes.c_double(snrl_db), ctypes.c_double(pnorm), _d(u),
                             rho.size, _d(rho), ctypes.c_double(a), ctypes.c_double(c),
                             _d(h), uc, _d(terms), _d(gu), _d(gr))
    return terms, gu, gr


def project_thresholds(rho):
    """Nearest ordered set 0 <= rho_0 <= ... <= rho_{K-1} <= 1 (returns a copy)."""
    r = _f64(rho).copy()
    lib().or_project_thresholds(r.size, _d(r))
    return r


def sqngd_outer_rho(state, cfg):
    """One outer iteration of Algorithm 1 with trainable thresholds; state holds
    float64 u, h, mu, vu, mh, vh, rho, mr, vr and counters t_x, t_h (in place)."""
    M, N = state["u"].shape
    nu, w = _grid(cfg["nu"], cfg["k_lo"], cfg["k_hi"], cfg.get("weights"))
    n_ev = cfg["n_h"] + cfg["n_x"]
    losses = np.zeros(n_ev)
    wpsl = np.zeros(n_ev)
    tx = ctypes.c_longlong(state["t_x"])
    th = ctypes.c_longlong(state["t_h"])
    for k in ("rho", "mr", "vr"):
        assert state[k].dtype == np.float64 and state[k].flags.c_contiguous
    lib().or_sqngd_outer_rho(
        M, N, nu.size, _d(nu), cfg["k_lo"], cfg["k_hi"], _d(w), ctypes.c_double(cfg["eps"]),
        ctypes.c_double(cfg["snrl_db"]), ctypes.c_double(cfg.get("pnorm", 0.0)),
        cfg["B"], state["rho"].size, _d(state["rho"]), ctypes.c_double(cfg["a"]), ctypes.c_double(cfg["c"]),
        cfg["n_h"], cfg["n_x"], ctypes.c_double(cfg["lr_h"]), ctypes.c_double(cfg["lr_x"]),
        ctypes.c_double(cfg["lr_rho"]), ctypes.c_double(cfg.get("b1", 0.9)),
        ctypes.c_double(cfg.get("b2", 0.999)), ctypes.c_double(cfg.get("adam_eps", 1e-8)),
        _d(state["u"]), _d(state["h"].view(np.float64)), _d(state["mu"]), _d(state["vu"]),
        _d(state["mh"].view(np.float64)), _d(state["vh"].view(np.float64)), _d(state["mr"]), _d(state["vr"]),
        ctypes.byref(tx), ctypes.byref(th), _d(losses), _d(wpsl))
    state["t_x"] = tx.value
    state["t_h"] = th.value
    return losses, wpsl


# ---------------------------------------------------------------- SQNAF (h = x)
def grad_matched(x, nu, k_lo, k_hi, weights=None, eps=0.1, snrl_db=0.5, pnorm=0.0, use_cell=None):
    """Loss L(x, x) and its total gradient when every filter is its waveform
    (SQNAF, Section IV); returns (terms, g)."""
    x = _c128(x)
    M, N = x.shape
    nu, w = _grid(nu, k_lo, k_hi, weights)
    terms = np.zeros(6)
    g = np.zeros_like(x)
    uc = None if use_cell is None else (ctypes.c_longlong * 1)(int(use_cell))
    lib().or_grad_matched(M, N, nu.size, _d(nu), k_lo, k_hi, _d(w), ctypes.c_double(eps),
                          ctypes.c_double(snrl_db), ctypes.c_double(pnorm), _d(x), uc, _d(terms), _d(g))
    return terms, g


def loss_grad_u_matched(u, rho, a, c, nu, k_lo, k_hi, weights=None, eps=0.1, snrl_db=0.5,
                        pnorm=0.0, use_cell=None):
    """SQNAF loss of the soft waveform and its gradient w.r.t. the logits."""
    u = _f64(u)
    M, N = u.shape
    nu, w = _grid(nu, k_lo, k_hi, weights)
    terms = np.zeros(6)
    gu = np.zeros((M, N))
    uc = None if use_cell is None else (ctypes.c_longlong * 1)(int(use_cell))
    lib().or_loss_grad_u_matched(M, N, nu.size, _d(nu), k_lo, k_hi, _d(w), ctypes.c_double(eps),
                                 ctypes.c_double(snrl_db), ctypes.c_double(pnorm), _d(u),
                                 rho.size, _d(_f64(rho)), ctypes.c_double(a), ctypes.c_double(c),
                                 uc, _d(terms), _d(gu))
    return terms, gu


def sqnaf_outer(state, cfg):
    """One outer iteration of SQNAF (Step A skipped, the hard design scored
    first); state holds float64 u, mu, vu and t_x, updated in place.
    Returns the 1 + n_x losses and L_WPSL values."""
    M, N = state["u"].shape
    nu, w = _grid(cfg["nu"], cfg["k_lo"], cfg["k_hi"], cfg.get("weights"))
    rho = _f64(cfg["rho"])
    n_ev = 1 + cfg["n_x"]
    losses = np.zeros(n_ev)
    wpsl = np.zeros(n_ev)
    tx = ctypes.c_longlong(state["t_x"])
    lib().or_sqnaf_outer(
        M, N, nu.size, _d(nu), cfg["k_lo"], cfg["k_hi"], _d(w), ctypes.c_double(cfg["eps"]),
        ctypes.c_double(cfg["snrl_db"]), ctypes.c_double(cfg.get("pnorm", 0.0)),
        cfg["B"], rho.size, _d(rho), ctypes.c_double(cfg["a"]), ctypes.c_double(cfg["c"]),
        cfg["n_x"], ctypes.c_double(cfg["lr_x"]), ctypes.c_double(cfg.get("b1", 0.9)),
        ctypes.c_double(cfg.get("b2", 0.999)), ctypes.c_double(cfg.get("adam_eps", 1e-8)),
        _d(state["u"]), _d(state["mu"]), _d(state["vu"]), ctypes.byref(tx), _d(losses), _d(wpsl))
    state["t_x"] = tx.value
    return losses, wpsl


def stop_rule(wpsl, patience, t_max, best_wpsl=float("inf"), best_outer=-1, t0=0):
    """Algorithm 1's stopping test (Section III-C): training ends when further
    outer iterations bring no improvement in the WPSL, or after T outer
    iterations.  Read as: wpsl[i] is the hard design's L_WPSL scored by outer
    iteration t0 + i; an iteration improves when its value is strictly below
    the best so far; the run stops after iteration t once t - (iteration of
    the best) >= patience (a fresh record counts from t0 - 1), or at t_max.
    Returns (iterations run, 1 patience / 2 t_max / 0 the sequence ran out,
    best value, its iteration)."""
    if best_outer < 0:
        best_outer = t0 - 1
    t = t0
    for v in wpsl:
        if t >= t_max:
            return t - t0, 2, best_wpsl, best_outer
        if v < best_wpsl:
            best_wpsl, best_outer = v, t
        if t - best_outer >= patience:
            return t + 1 - t0, 1, best_wpsl, best_outer
        t += 1
    return t - t0, (2 if t >= t_max else 0), best_wpsl, best_outer


def metrics(x, h, nu, k_lo, k_hi, weights=None):
    """(APSL dB, CPSL dB, PSLR dB, max SNRL dB) and per-waveform SNRL (Eqs. 10, 48)."""
    x, h = _c128(x), _c128(h)
    M, N = x.shape
    nu, w = _grid(nu, k_lo, k_hi, weights)
    out = np.zeros(4)
    snrl = np.zeros(M)
    lib().or_metrics(M, N, nu.size, _d(nu), k_lo, k_hi, _d(w), _d(x), _d(h), _d(out), _d(snrl))
    return out, snrl


def init_logits(b, B, r_n):
    """Initial logits for phase indices b (middle copy of the K = B*r_n
    quantization regions, so the hard quantizer returns q = r_n//2 * B + b)."""
    K = B * r_n
    z0 = ((r_n // 2) * B + np.asarray(b, dtype=np.float64)) / K
    return np.log(z0 / (1.0 - z0))


def grad_at_cell(x, h, nu, k_lo, k_hi, cell, w_cell, eps=0.1, snrl_db=0.5):
    """Gradient with the exact max taken at `cell` (weight w_cell), no grid
    scan; returns (chi at the cell, gx, gh)."""
    x, h = _c128(x), _c128(h)
    M, N = x.shape
    nu = _f64(nu)
    gx = np.zeros_like(x)
    gh = np.zeros_like(h)
    chi = np.zeros(2)
    lib().or_grad_at_cell(M, N, nu.size, _d(nu), k_lo, k_hi, ctypes.c_double(w_cell),
                          ctypes.c_double(eps), ctypes.c_double(snrl_db), _d(x), _d(h),
                          ctypes.c_longlong(int(cell)), _d(chi), _d(gx), _d(gh))
    return chi[0] + 1j * chi[1], gx, gh
