"""bench.py's roofline arithmetic and traffic records, on CPU: the algorithmic
FLOP counts against explicit enumeration of the work each kernel must do."""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2604_25728_gb300 import workloads as wl  # noqa: E402


def _valid_products(w):
    return sum(max(0, w.N - abs(k)) for k in range(w.k_lo, w.k_hi + 1))


def test_fft_flops_by_enumeration():
    for w in (wl.tiny(), wl.mid(), wl.small(3, 50, 4, 32, -10, 30)):
        P, rows = w.M * w.M, w.M * w.M * w.D
        exp = 6 * P * _valid_products(w) + rows * 5 * w.L * math.log2(w.L) + 3 * rows * w.L
        assert abs(bench._fwd_flops(w) - exp) < 1e-6 * exp
    assert abs(bench._fwd_flops(wl.mid()) - 427425792.0) < 1.0


def test_split_and_correlation_flops_by_enumeration():
    w = wl.precision()
    assert bench._split_flops(w) == 3 * 8 * w.M * w.M * _valid_products(w) * w.L
    c = wl.correlation()
    assert _valid_products(c) == c.N * c.N                 # every delay: sum (N - |k|) = N^2
    assert bench._corr_flops(c) == 8 * 4 * c.N * c.N + 3 * 4 * c.D


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    h = bench._source_hash(bench.FWD_SOURCES)
    assert h == bench._source_hash(bench.FWD_SOURCES) and len(h) == 16
    rec = {"source_hash": h, "dram_bytes_per_launch": 1234}
    (tmp_path / "t.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench._traffic_record(h, "t.json") == 1234
    assert bench._traffic_record("0" * 16, "t.json") is None      # sources changed since the capture
    assert bench._traffic_record(h, "missing.json") is None


def test_committed_traffic_records_name_their_commands():
    for name in ("fwd_fft_mid_traffic.json", "fwd_gemm_precision_traffic.json", "fwd_fft_differentiation_traffic.json"):
        rec = json.load(open(os.path.join(ROOT, "profiles", name)))
        assert rec["command"].startswith("ncu ") and "--clock-control none" in rec["command"]
        assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]


def test_table6_settings_follow_the_paper():
    """The optimisation-time settings (Table VI): M x N x B over {2, 10} x
    {512, 1200} x {4, 16}, |k| <= 50, f in [-0.5, 0.5] cycles per waveform
    (|nu| <= 0.5/N per chip, end points included), SNRL target 0.5 dB, and the
    Section IV hyper-parameters N_h = N_x = 10, eta_h = 5e-2, eps = 0.1."""
    from paper_2604_25728_gb300 import generator
    ws = generator.table6_settings(bins=64)
    assert sorted((w.M, w.N, w.B) for w in ws) == sorted(
        (M, N, B) for M in (2, 10) for N in (512, 1200) for B in (4, 16))
    for w in ws:
        assert (w.k_lo, w.k_hi, w.L) == (-50, 50, 64)
        assert abs(w.nu[0] * w.N + 0.5) < 1e-15 and abs(w.nu[-1] * w.N - 0.5) < 1e-15
        assert all(w.nu[i] < w.nu[i + 1] for i in range(w.L - 1))
        assert (w.snrl_db, w.n_h, w.n_x, w.lr_h, w.eps) == (0.5, 10, 10, 5e-2, 0.1)


def test_dump_bytes_by_enumeration():
    """The materialising forward writes one complex64 per (pair, delay, bin)
    and reads the complex64 waveforms and filters once."""
    for w in (wl.tiny(), wl.mid(), wl.small(3, 50, 4, 32, -10, 30)):
        cells = sum(1 for _m in range(w.M) for _l in range(w.M) for _k in range(w.k_lo, w.k_hi + 1)
                    for _j in range(w.L))
        assert bench._dump_bytes(w) == 8 * cells + 8 * 2 * w.M * w.N


def test_paper_fft_formulation_matches_the_oracle():
    """The library-FFT comparator (the paper's Doppler-major formulation, run
    here by torch.fft on the CPU) computes Eq. 6 and the maxima of Eqs. 8-9:
    against the oracle on a small grid with a delay window that is not
    centred and an offset Doppler grid."""
    import numpy as np
    import torch
    import oracle as orc
    M, N, L, k_lo, k_hi = 3, 40, 16, -12, 25
    nu = wl.full_grid(L) + 0.01
    x = wl.unit_phasors(3, M, N)
    h = wl.complex_normal(4, M, N)
    chi, wapsl, wcpsl = bench.paper_fft_wpsl(torch.from_numpy(x.astype(np.complex64)),
                                             torch.from_numpy(h.astype(np.complex64)), nu, k_lo, k_hi, 1.0 / N)
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi)
    assert np.max(np.abs(chi.numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))
    r = orc.loss(x, h, nu, k_lo, k_hi)
    assert abs(float(wapsl) - r["wapsl"]) <= 1e-5 * r["wapsl"]
    assert abs(float(wcpsl) - r["wcpsl"]) <= 1e-5 * r["wcpsl"]


def test_oracle_sample_share_by_enumeration():
    """The reference sample (the delay window |k| <= 63 of the workload)
    counts as its share of the lag products: enumerated pair by pair."""
    w = wl.differentiation()
    win = sum(w.N - abs(k) for k in range(-63, 64))
    full = sum(w.N - abs(k) for k in range(w.k_lo, w.k_hi + 1))
    assert full == w.N * w.N
    assert abs(bench.sample_share(w) - win / full) < 1e-15
    s = bench._oracle_window(w)
    assert (s.k_lo, s.k_hi, s.M, s.N, s.L) == (-63, 63, w.M, w.N, w.L)


def test_fp32_peak_from_unit_counts():
    peak, note = bench._fp32_peak_tflops(sms=152, mhz=2070.0)
    assert abs(peak - 152 * 128 * 2 * 2.070e9 / 1e12) < 1e-9 and "152 SMs" in note


def test_adjoint_flops_by_enumeration():
    """Per row of the winning class: two L-point transforms, 6 per cell (|chi|^2
    and g) and 22 per valid lag product (the recomputed product and the two
    gradient accumulations)."""
    w = wl.small(2, 40, 4, 32, -10, 30)
    valid = _valid_products(w)
    rows = w.M * w.D
    exp = rows * (2 * 5 * w.L * math.log2(w.L) + 6 * w.L) + 22 * valid * rows / w.D
    assert abs(bench._adj_flops(w, rows) - exp) < 1e-9 * exp


def test_clock_samples_before_the_timed_region_are_dropped():
    """Only samples taken after mark() count; throttle reasons are read from
    the Active columns."""
    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc = _Proc()
    idle = "0, 345, 2070, 100.0, 0x1, Not Active, Not Active, Not Active, Not Active"
    busy = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    s.lines = [idle, idle]
    s.mark()
    s.lines += [busy, busy, capped]
    r = s.stop()
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
