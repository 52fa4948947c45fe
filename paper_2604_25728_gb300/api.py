"""Python binding of the SQNGD C ABI (argument marshalling only).

Every method forwards device pointers of torch tensors to the entry point of
the same name in libsqngd.so; all arithmetic runs in the library's sm_103a
kernels.  PyTorch provides device memory and the stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import AF_PATH_AUTO, AF_PATH_DFT, AF_PATH_FFT, AF_PATH_SPLIT_BF16, AF_TERMS_FIXED, AfError  # noqa: F401


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, shape, name):
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")


class Context:
    """One af_ctx: problem sizes, grid, loss and optimiser constants."""

    def __init__(self, M, N, B, nu, k_lo, k_hi, weights=None, eps=0.1, snrl_db=0.5, r_n=100,
                 c=300.0, pnorm=0.0, path=AF_PATH_AUTO, n_h=10, n_x=10, lr_h=5e-2, lr_x=5e-4,
                 beta1=0.9, beta2=0.999, adam_eps=1e-8, matched=False, train_rho=False, lr_rho=1e-5,
                 device=None, stream=None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.M, self.N, self.B = int(M), int(N), int(B)
        self.nu = np.ascontiguousarray(nu, dtype=np.float64)
        self.L = int(self.nu.size)
        self.k_lo, self.k_hi = int(k_lo), int(k_hi)
        self.D = self.k_hi - self.k_lo + 1
        self.r_n, self.c = int(r_n), float(c)
        self.K = self.B * self.r_n
        self.n_h, self.n_x = int(n_h), int(n_x)
        self.matched = bool(matched)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        if w is not None and w.shape != (self.D, self.L):
            raise ValueError(f"weights must be [D, L] = [{self.D}, {self.L}]")
        cfg = _lib.AfConfig(
            M=self.M, N=self.N, B=self.B, L=self.L,
            nu=self.nu.ctypes.data_as(_lib.P_double), k_lo=self.k_lo, k_hi=self.k_hi,
            weights=None if w is None else w.ctypes.data_as(_lib.P_float),
            eps=float(eps), snrl_db=float(snrl_db), r_n=self.r_n, c=self.c, pnorm=float(pnorm),
            path=int(path), n_h=self.n_h, n_x=self.n_x, lr_h=float(lr_h), lr_x=float(lr_x),
            beta1=float(beta1), beta2=float(beta2), adam_eps=float(adam_eps), matched=int(self.matched),
            train_rho=int(bool(train_rho)), lr_rho=float(lr_rho))
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            handle = ctypes.c_void_p()
            st = self.lib.af_init(ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle))
            _lib.check(st, None)
        self.handle = handle

    # -------------------------------------------------------------- helpers
    def close(self):
        if getattr(self, "handle", None):
            self.lib.af_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        _lib.check(st, self.handle)

    @property
    def path(self) -> int:
        return int(self.lib.af_path_of(self.handle))

    def _mn(self, t, name, complex_=False):
        _need(t, torch.complex64 if complex_ else torch.float32, (self.M, self.N), name)
        return t

    def empty_terms(self):
        return torch.empty(AF_TERMS_FIXED + self.M, dtype=torch.float64, device=self.device)

    # ------------------------------------------------------------ entry points
    def af_sync(self):
        self._check(self.lib.af_sync(self.handle))

    def af_set_thresholds(self, rho):
        r = np.ascontiguousarray(rho, dtype=np.float32)
        if r.size != self.K:
            raise ValueError(f"need K = {self.K} thresholds")
        self._check(self.lib.af_set_thresholds(self.handle, r.ctypes.data_as(_lib.P_float)))

    def af_ambiguity(self, x, h, chi=None):
        self._mn(x, "x", True); self._mn(h, "h", True)
        if chi is None:
            chi = torch.empty((self.M, self.M, self.D, self.L), dtype=torch.complex64, device=self.device)
        _need(chi, torch.complex64, (self.M, self.M, self.D, self.L), "chi")
        self._check(self.lib.af_ambiguity(self.handle, _ptr(x), _ptr(h), _ptr(chi)))
        return chi

    def af_forward(self, x, h):
        self._mn(x, "x", True); self._mn(h, "h", True)
        self._check(self.lib.af_forward(self.handle, _ptr(x), _ptr(h)))

    def _filters(self, h):
        """Filters argument: ignored by matched (SQNAF) contexts, which may pass None."""
        if h is None and self.matched:
            return None
        return self._mn(h, "h", True)

    def af_loss_grad_xh(self, x, h, terms=None, grad_x=None, grad_h=None):
        self._mn(x, "x", True); h = self._filters(h)
        terms = self.empty_terms() if terms is None else terms
        self._check(self.lib.af_loss_grad_xh(self.handle, _ptr(x), _ptr(h), _ptr(terms), _ptr(grad_x), _ptr(grad_h)))
        return terms, grad_x, grad_h

    def af_loss_grad(self, u, h, use_hard=False, terms=None, grad_u=None, grad_h=None):
        self._mn(u, "u"); h = self._filters(h)
        terms = self.empty_terms() if terms is None else terms
        self._check(self.lib.af_loss_grad(self.handle, _ptr(u), _ptr(h), int(bool(use_hard)), _ptr(terms),
                                          _ptr(grad_u), _ptr(grad_h)))
        return terms, grad_u, grad_h

    def af_loss_grad_rho(self, u, h, terms=None, grad_u=None, grad_h=None, grad_rho=None):
        """Loss and gradients through the soft chain, with dL/drho (Eq. 24)."""
        self._mn(u, "u"); h = self._filters(h)
        terms = self.empty_terms() if terms is None else terms
        grad_rho = torch.empty(self.K, dtype=torch.float32, device=self.device) if grad_rho is None else grad_rho
        self._check(self.lib.af_loss_grad_rho(self.handle, _ptr(u), _ptr(h), _ptr(terms), _ptr(grad_u),
                                              _ptr(grad_h), _ptr(grad_rho)))
        return terms, grad_u, grad_h, grad_rho

    def attach_generator(self, rn, y0):
        """Train the transmit generator rn (ResNetGenerator) in Step B instead of
        the logits; y0 [M N] float32 on the device; rn = None detaches."""
        if rn is not None:
            _need(y0, torch.float32, (self.M * self.N,), "y0")
        self._generator = (rn, y0)          # keep both alive while attached
        self._check(self.lib.sqngd_attach_generator(self.handle, None if rn is None else rn.handle,
                                                    None if rn is None else _ptr(y0)))

    def af_get_thresholds(self):
        r = np.zeros(self.K, dtype=np.float32)
        self._check(self.lib.af_get_thresholds(self.handle, r.ctypes.data_as(_lib.P_float)))
        return r

    def af_project_thresholds(self, rho):
        _need(rho, torch.float32, (self.K,), "rho")
        self._check(self.lib.af_project_thresholds(self.handle, _ptr(rho)))
        return rho

    def quantize(self, z, q=None, x=None):
        n = z.numel()
        q = torch.empty(z.shape, dtype=torch.int32, device=self.device) if q is None else q
        x = torch.empty(z.shape, dtype=torch.complex64, device=self.device) if x is None else x
        self._check(self.lib.quantize(self.handle, _ptr(z), n, _ptr(q), _ptr(x)))
        return q, x

    def soft_quantize(self, z, y=None, dydz=None, x=None):
        n = z.numel()
        y = torch.empty_like(z) if y is None else y
        dydz = torch.empty_like(z) if dydz is None else dydz
        x = torch.empty(z.shape, dtype=torch.complex64, device=self.device) if x is None else x
        self._check(self.lib.soft_quantize(self.handle, _ptr(z), n, _ptr(y), _ptr(dydz), _ptr(x)))
        return y, dydz, x

    def af_project(self, h):
        self._mn(h, "h", True)
        self._check(self.lib.af_project(self.handle, _ptr(h)))
        return h

    def sqngd_init(self, b, noise=None, u=None, h=None):
        _need(b, torch.int32, (self.M, self.N), "b")
        u = torch.empty((self.M, self.N), dtype=torch.float32, device=self.device) if u is None else u
        h = torch.empty((self.M, self.N), dtype=torch.complex64, device=self.device) if h is None else h
        self._check(self.lib.sqngd_init(self.handle, _ptr(b), _ptr(noise), _ptr(u), _ptr(h)))
        return u, h

    def sqngd_step(self, state: "SqngdState", n_outer: int, log: bool = True):
        cs = state.c_struct()
        buf = None
        if log:
            evals = (1 + self.n_x) if self.matched else (self.n_h + self.n_x)
            buf = np.zeros((n_outer, evals, 4), dtype=np.float64)
        self._check(self.lib.sqngd_step(self.handle, ctypes.byref(cs), int(n_outer),
                                        None if buf is None else buf.ctypes.data_as(_lib.P_double)))
        state.t_h, state.t_x, state.outer = cs.t_h, cs.t_x, cs.outer
        return buf

    def sqngd_run(self, state: "SqngdState", t_max: int, patience: int = 50, log: bool = True):
        """Outer iterations until Algorithm 1's stopping test fires (no better
        hard WPSL for `patience` iterations) or state.outer reaches t_max.
        Returns (log [n_done, evals, 4] or None, the stopped code: 1 patience,
        2 t_max).  The rule's record lives in state.stop (kept by save/load)."""
        cs = state.c_struct()
        stop = _lib.AfStop(best_wpsl=float(state.stop[0]), best_outer=int(state.stop[1]), stopped=0)
        evals = (1 + self.n_x) if self.matched else (self.n_h + self.n_x)
        rows = max(0, int(t_max) - int(state.outer))
        buf = np.zeros((rows, evals, 4), dtype=np.float64) if log else None
        done = ctypes.c_int64(0)
        self._check(self.lib.sqngd_run(self.handle, ctypes.byref(cs), int(t_max), int(patience), ctypes.byref(stop),
                                       None if buf is None else buf.ctypes.data_as(_lib.P_double),
                                       ctypes.byref(done)))
        state.t_h, state.t_x, state.outer = cs.t_h, cs.t_x, cs.outer
        state.stop = [stop.best_wpsl, stop.best_outer]
        return (None if buf is None else buf[:done.value]), int(stop.stopped)

    def get_rho_state(self):
        """(rho, m_rho, v_rho, uniform) of the quantization thresholds."""
        r, m, v = (np.zeros(self.K, dtype=np.float32) for _ in range(3))
        uni = ctypes.c_int32(0)
        self._check(self.lib.af_get_rho_state(self.handle, r.ctypes.data_as(_lib.P_float),
                                              m.ctypes.data_as(_lib.P_float), v.ctypes.data_as(_lib.P_float),
                                              ctypes.byref(uni)))
        return r, m, v, int(uni.value)

    def set_rho_state(self, rho, m_rho, v_rho, uniform: int):
        r, m, v = (np.ascontiguousarray(a, dtype=np.float32) for a in (rho, m_rho, v_rho))
        if not (r.size == m.size == v.size == self.K):
            raise ValueError(f"need K = {self.K} thresholds and moments")
        self._check(self.lib.af_set_rho_state(self.handle, r.ctypes.data_as(_lib.P_float),
                                              m.ctypes.data_as(_lib.P_float), v.ctypes.data_as(_lib.P_float),
                                              int(uniform)))

    def af_eval_hard(self, u, h):
        self._mn(u, "u"); h = self._filters(h)
        out = np.zeros(4 + self.M, dtype=np.float64)
        self._check(self.lib.af_eval_hard(self.handle, _ptr(u), _ptr(h), out.ctypes.data_as(_lib.P_double)))
        return out


class ResNetGenerator:
    """rn_net: the transmit-side ResNet z = f_theta(y0) of Eq. 17 for P = M N
    phases (include/resnet.h); forward gives the pre-sigmoid output u."""

    def __init__(self, P: int, device=None, stream=None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.P = int(P)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            handle = ctypes.c_void_p()
            st = self.lib.rn_create(self.P, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle))
            self._check(st, None)
        self.handle = handle

    @staticmethod
    def param_count(P: int) -> int:
        return int(_lib.load().rn_param_count(int(P)))

    def _check(self, st, handle):
        if st != _lib.AF_OK:
            msg = self.lib.rn_last_error(handle).decode() if handle is not None else ""
            raise AfError(st, msg)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != self.param_count(self.P):
            raise ValueError("wrong parameter count")
        self._check(self.lib.rn_set_params(self.handle, t.ctypes.data_as(_lib.P_float)), self.handle)

    def get_params(self):
        t = np.zeros(self.param_count(self.P), dtype=np.float32)
        self._check(self.lib.rn_get_params(self.handle, t.ctypes.data_as(_lib.P_float)), self.handle)
        return t

    def get_adam(self):
        """The Adam moments (m, v) of every parameter."""
        m = np.zeros(self.param_count(self.P), dtype=np.float32)
        v = np.zeros_like(m)
        self._check(self.lib.rn_get_adam(self.handle, m.ctypes.data_as(_lib.P_float),
                                         v.ctypes.data_as(_lib.P_float)), self.handle)
        return m, v

    def set_adam(self, m, v):
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        if m.size != self.param_count(self.P) or v.size != m.size:
            raise ValueError("wrong moment count")
        self._check(self.lib.rn_set_adam(self.handle, m.ctypes.data_as(_lib.P_float),
                                         v.ctypes.data_as(_lib.P_float)), self.handle)

    def forward(self, y0, u=None):
        _need(y0, torch.float32, (self.P,), "y0")
        u = torch.empty(self.P, dtype=torch.float32, device=self.device) if u is None else u
        self._check(self.lib.rn_forward(self.handle, _ptr(y0), _ptr(u)), self.handle)
        return u

    def train_step(self, y0, du, lr: float, t: int, u=None):
        _need(y0, torch.float32, (self.P,), "y0")
        _need(du, torch.float32, (self.P,), "du")
        u = torch.empty(self.P, dtype=torch.float32, device=self.device) if u is None else u
        self._check(self.lib.rn_train_step(self.handle, _ptr(y0), _ptr(du), float(lr), int(t), _ptr(u)),
                    self.handle)
        return u


@dataclass
class SqngdState:
    """Device buffers of the optimiser state (caller-owned, see af_state)."""
    u: torch.Tensor
    h: Optional[torch.Tensor]
    m_u: torch.Tensor
    v_u: torch.Tensor
    m_h: Optional[torch.Tensor]
    v_h: Optional[torch.Tensor]
    best_q: torch.Tensor
    best_h: torch.Tensor
    best: torch.Tensor
    t_h: int = 0
    t_x: int = 0
    outer: int = 0
    # record of the stopping rule (sqngd_run): best hard WPSL so far and its outer iteration
    stop: list = field(default_factory=lambda: [float("inf"), -1])

    @classmethod
    def create(cls, u, h=None):
        """h = None: matched (SQNAF) state, no filters and no filter moments."""
        z = torch.zeros_like
        best = torch.tensor([float("inf"), float("inf"), -1.0, float("inf")], dtype=torch.float64,
                            device=u.device)
        best_h = torch.zeros(u.shape, dtype=torch.complex64, device=u.device) if h is None else h.clone()
        return cls(u=u, h=h, m_u=z(u), v_u=z(u), m_h=None if h is None else z(h), v_h=None if h is None else z(h),
                   best_q=torch.zeros(u.shape, dtype=torch.int32, device=u.device), best_h=best_h,
                   best=best)

    _BUFFERS = ("u", "h", "m_u", "v_u", "m_h", "v_h", "best_q", "best_h", "best")

    def save(self, path: str, ctx: Optional["Context"] = None, generator: Optional["ResNetGenerator"] = None):
        """Checkpoint every buffer of the state, the step counters and the
        stopping-rule record to an .npz file; with `ctx`, also the context's
        threshold state (rho, its Adam moments, uniform flag); with
        `generator`, the attached generator's parameters and Adam moments."""
        arrays = {k: getattr(self, k).detach().cpu().numpy() for k in self._BUFFERS if getattr(self, k) is not None}
        if ctx is not None:
            r, m, v, uni = ctx.get_rho_state()
            arrays.update(rho=r, m_rho=m, v_rho=v, rho_uniform=np.int32(uni))
        if generator is not None:
            gm, gv = generator.get_adam()
            arrays.update(gen_theta=generator.get_params(), gen_m=gm, gen_v=gv)
        np.savez(path, t_h=np.int64(self.t_h), t_x=np.int64(self.t_x), outer=np.int64(self.outer),
                 stop_best=np.float64(self.stop[0]), stop_outer=np.int64(self.stop[1]), **arrays)

    @classmethod
    def load(cls, path: str, device=None, ctx: Optional["Context"] = None,
             generator: Optional["ResNetGenerator"] = None, y0=None):
        """The state saved by `save`, with its buffers on `device`; with `ctx`
        and `generator`, their saved parts are restored into them (the file
        must hold them).  A generator's next training step uses the
        activations of its last forward pass, so with `generator` pass its
        input y0 as well: the forward pass is rerun at the restored
        parameters."""
        with np.load(path) as f:
            t = {k: (torch.from_numpy(f[k]).to(device) if k in f.files else None) for k in cls._BUFFERS}
            stop = [float(f["stop_best"]), int(f["stop_outer"])] if "stop_best" in f.files else [float("inf"), -1]
            if ctx is not None:
                ctx.set_rho_state(f["rho"], f["m_rho"], f["v_rho"], int(f["rho_uniform"]))
            if generator is not None:
                if y0 is None:
                    raise ValueError("restoring a generator needs its input y0")
                generator.set_params(f["gen_theta"])
                generator.set_adam(f["gen_m"], f["gen_v"])
                generator.forward(y0)
            return cls(**t, t_h=int(f["t_h"]), t_x=int(f["t_x"]), outer=int(f["outer"]), stop=stop)

    def c_struct(self):
        p = lambda t: 0 if t is None else t.data_ptr()
        return _lib.AfState(u_dev=p(self.u), h_dev=p(self.h), m_u_dev=p(self.m_u),
                            v_u_dev=p(self.v_u), m_h_dev=p(self.m_h), v_h_dev=p(self.v_h),
                            best_q_dev=p(self.best_q), best_h_dev=p(self.best_h),
                            best_dev=p(self.best), t_h=self.t_h, t_x=self.t_x, outer=self.outer)


class AfLoss(torch.autograd.Function):
    """Loss of Eq. 42 through the soft transmit chain as a
    torch.autograd.Function.  The forward pass evaluates the loss alone (no
    adjoint, no gradient buffers) and keeps only u and h; the backward pass
    calls the library again with gradient outputs, so the hand-written
    adjoint recomputes the products and spectra it needs instead of storing
    them, and scales its gradient by the incoming one."""

    @staticmethod
    def forward(fctx, u, h, ctx: Context):
        u_, h_ = u.detach().contiguous(), h.detach().contiguous()
        terms, _, _ = ctx.af_loss_grad(u_, h_, False)
        fctx.save_for_backward(u_, h_)
        fctx.af_ctx = ctx
        return terms[0].clone()

    @staticmethod
    def backward(fctx, g):
        u, h = fctx.saved_tensors
        gu = torch.empty_like(u)
        gh = torch.empty_like(h)
        fctx.af_ctx.af_loss_grad(u, h, False, grad_u=gu, grad_h=gh)
        s = g.to(torch.float32)
        return gu * s, gh * s, None


# ------------------------------------------------------------ warm start --
def ws_cond(M: int, N: int, B: int, window: float, kmax: int):
    """The five conditioning scalars of the warm-start network for a problem
    of M waveforms of N chips, B levels, Doppler half-width `window`
    (cycles/chip) and delay half-width `kmax`."""
    return [M / 8.0, N / 1024.0, B / 64.0, 10.0 * float(window), float(kmax) / N]


class WarmStart:
    """One ws_net: the warm-start network's FP16/FP32 parameters, Adam state
    and activations for up to batch_max designs of up to n_max chips."""

    def __init__(self, batch_max: int, n_max: int, device=None, stream=None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.batch_max, self.n_max = int(batch_max), int(n_max)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            handle = ctypes.c_void_p()
            st = self.lib.ws_create(self.batch_max, self.n_max, ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(handle))
            self._check(st, None)
        self.handle = handle

    @staticmethod
    def param_count() -> int:
        return int(_lib.load().ws_param_count())

    def _check(self, st, handle):
        if st != _lib.AF_OK:
            msg = self.lib.ws_last_error(handle).decode() if handle is not None else ""
            raise AfError(st, msg)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.ws_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.param_count():
            raise ValueError(f"expected {self.param_count()} parameters, got {p.size}")
        self._check(self.lib.ws_set_params(self.handle, p.ctypes.data_as(_lib.P_float)), self.handle)

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.param_count(), dtype=np.float32)
        self._check(self.lib.ws_get_params(self.handle, p.ctypes.data_as(_lib.P_float)), self.handle)
        return p

    @staticmethod
    def _cfg(M, N, B, cond):
        c = _lib.WsConfig(M=int(M), N=int(N), B=int(B))
        for i in range(5):
            c.cond[i] = float(cond[i])
        return c

    def forward(self, b0, B, cond, logits=True):
        """b0: int32 [batch, M, N] on the device.  Returns (logits [batch, 64, N]
        or None, b [batch, M, N] int32)."""
        batch, M, N = b0.shape
        _need(b0, torch.int32, (batch, M, N), "b0")
        cfg = self._cfg(M, N, B, cond)
        lg = torch.empty((batch, 64, N), dtype=torch.float32, device=b0.device) if logits else None
        b = torch.empty((batch, M, N), dtype=torch.int32, device=b0.device)
        self._check(self.lib.ws_forward(self.handle, ctypes.byref(cfg), int(batch), _ptr(b0), _ptr(lg), _ptr(b)),
                    self.handle)
        return lg, b

    def loss_grad(self, b0, target, B, cond):
        batch, M, N = b0.shape
        _need(target, torch.int32, (batch, M, N), "target")
        cfg = self._cfg(M, N, B, cond)
        loss = ctypes.c_double()
        g = np.zeros(self.param_count(), dtype=np.float32)
        self._check(self.lib.ws_loss_grad(self.handle, ctypes.byref(cfg), int(batch), _ptr(b0), _ptr(target),
                                          ctypes.byref(loss), g.ctypes.data_as(_lib.P_float)), self.handle)
        return loss.value, g

    def train_step(self, b0, target, B, cond, lr: float, sync: bool = True):
        batch, M, N = b0.shape
        _need(target, torch.int32, (batch, M, N), "target")
        cfg = self._cfg(M, N, B, cond)
        loss = ctypes.c_double()
        self._check(self.lib.ws_train_step(self.handle, ctypes.byref(cfg), int(batch), _ptr(b0), _ptr(target),
                                           float(lr), ctypes.byref(loss) if sync else None), self.handle)
        return loss.value if sync else None
