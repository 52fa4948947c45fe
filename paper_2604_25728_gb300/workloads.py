"""Seeded synthetic workloads (shapes, grids and random draws only).

This module holds the random inputs and problem sizes shared by the tests,
the benchmark and the oracle checks.  It contains none of the method's
arithmetic: no ambiguity function, loss, quantizer or optimiser step.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state advances by the golden
gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
published two-multiply finaliser.  Uniform doubles take the top 53 bits.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """`count` outputs of SplitMix64 started at state seed + stream * 2^32."""
    with np.errstate(over="ignore"):
        start = np.uint64((int(seed) + (int(stream) << 32)) & 0xFFFFFFFFFFFFFFFF)
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = start + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1)."""
    return (splitmix64(seed, count, stream) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Standard normal doubles (Box-Muller on two SplitMix64 streams)."""
    u1 = uniform(seed, count, 2 * stream + 1)
    u2 = uniform(seed, count, 2 * stream + 2)
    u1 = np.maximum(u1, 2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def phase_indices(seed: int, M: int, N: int, B: int) -> np.ndarray:
    """Uniform discrete phase indices b in [0, B), shape [M, N] (int32)."""
    u = uniform(seed, M * N, stream=7)
    return np.minimum((u * B).astype(np.int64), B - 1).astype(np.int32).reshape(M, N)


def complex_normal(seed: int, M: int, N: int, stream: int = 11) -> np.ndarray:
    """Circular complex Gaussian draws of unit variance per component, [M, N]."""
    re = normal(seed, M * N, stream)
    im = normal(seed, M * N, stream + 1)
    return (re + 1j * im).reshape(M, N)


def unit_phasors(seed: int, M: int, N: int, stream: int = 13) -> np.ndarray:
    """Random points on the unit circle (continuous phases), [M, N]."""
    return np.exp(2j * np.pi * uniform(seed, M * N, stream)).reshape(M, N)


def logits(seed: int, M: int, N: int, scale: float = 1.0, stream: int = 17) -> np.ndarray:
    """Random real logits (Gaussian, given scale), [M, N]."""
    return scale * normal(seed, M * N, stream).reshape(M, N)


def full_grid(L: int) -> np.ndarray:
    """L Doppler bins uniformly spanning nu in [-0.5, 0.5) cycles/chip."""
    return -0.5 + np.arange(L, dtype=np.float64) / L


def window_grid(W: float, L: int) -> np.ndarray:
    """L Doppler bins on the closed window [-W, W] (inclusive end points)."""
    return np.linspace(-W, W, L, dtype=np.float64)


@dataclass
class Workload:
    """One problem size: M waveforms of N chips, B phase levels, delays
    k_lo..k_hi and the Doppler grid nu (cycles/chip)."""
    name: str
    M: int
    N: int
    B: int
    k_lo: int
    k_hi: int
    nu: np.ndarray = field(repr=False)
    r_n: int = 100
    c: float = 300.0
    eps: float = 0.1
    snrl_db: float = 0.5
    n_h: int = 10
    n_x: int = 10
    lr_h: float = 5e-2
    lr_x: float = 5e-4

    @property
    def L(self) -> int:
        return int(self.nu.size)

    @property
    def D(self) -> int:
        return self.k_hi - self.k_lo + 1

    @property
    def K(self) -> int:
        return self.B * self.r_n


def tiny() -> Workload:
    """M=2, N=64, B=4, every delay, 64 bins over [-0.5, 0.5)."""
    return Workload("tiny M=2 N=64 B=4 L=64 full-range", 2, 64, 4, -63, 63, full_grid(64))


def mid() -> Workload:
    """M=4, N=512, B=16, every delay, 512 bins over [-0.5, 0.5)."""
    return Workload("mid M=4 N=512 B=16 L=512 full-range", 4, 512, 16, -511, 511, full_grid(512))


def precision() -> Workload:
    """M=8, N=1024, B=8, |k| <= 255, 64 bins on |nu| <= 0.05."""
    return Workload("precision M=8 N=1024 B=8 |k|<=255 L=64 |nu|<=0.05", 8, 1024, 8, -255, 255,
                    window_grid(0.05, 64))


def differentiation() -> Workload:
    """M=4, N=2048, B=64, every delay, 2048 bins over [-0.5, 0.5)."""
    return Workload("differentiation M=4 N=2048 B=64 L=2048 full-range", 4, 2048, 64, -2047, 2047,
                    full_grid(2048))


def learned() -> Workload:
    """M=4, N=1024, B=16, |k| <= 50, 128 bins on |nu| <= 0.1."""
    return Workload("learned M=4 N=1024 B=16 |k|<=50 L=128 |nu|<=0.1", 4, 1024, 16, -50, 50,
                    window_grid(0.1, 128))


def correlation() -> Workload:
    """Zero-Doppler correlation design: M=2, N=1200, B=16, every delay, the
    single bin nu = 0, SNRL target 0 dB (the setting of the paper's
    correlation comparison)."""
    return Workload("correlation M=2 N=1200 B=16 L=1 (nu=0) full-range", 2, 1200, 16, -1199, 1199,
                    np.zeros(1), snrl_db=0.0)


def small(M: int, N: int, B: int, L: int, k_lo: int | None = None, k_hi: int | None = None,
          r_n: int = 100) -> Workload:
    """A small full-grid case for parity tests."""
    k_lo = -(N - 1) if k_lo is None else k_lo
    k_hi = (N - 1) if k_hi is None else k_hi
    return Workload(f"small M={M} N={N} B={B} L={L}", M, N, B, k_lo, k_hi, full_grid(L), r_n=r_n)
