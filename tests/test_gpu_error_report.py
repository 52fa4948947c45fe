"""Per-workload error against the FP64 oracle, printed as one table row each
(run with -s to see them): |chi| error on sampled cells relative to the
mainlobe, PSL difference per class in dB, gradient error at the GPU's
winning cell relative to the largest gradient entry, and the optimiser's
loss+grad evaluations/s (sqngd_step, 20 evaluations per outer iteration).

Each row also asserts its path's bars: FP32 paths 1e-5 of the mainlobe and
0.05 dB, the split-BF16 path 1e-4 and 0.1 dB, gradients 1e-4.
"""

import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import api as a
    return a


def _pair(orc, seed, M, N, noise=0.3):
    x = wl.unit_phasors(seed, M, N).astype(np.complex64)
    h = orc.project(x.astype(np.complex128) + noise * wl.complex_normal(seed, M, N)).astype(np.complex64)
    return x, h


def _evals_per_s(api, ctx, w, seed, matched=False):
    b = torch.from_numpy(wl.phase_indices(seed, w.M, w.N, w.B)).cuda()
    u, h = ctx.sqngd_init(b)
    st = api.SqngdState.create(u, None if matched else h)
    ctx.sqngd_step(st, 2, log=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 10
    e0.record()
    ctx.sqngd_step(st, n, log=False)
    e1.record()
    e1.synchronize()
    ctx.af_sync()
    evals = (1 + w.n_x) if matched else (w.n_h + w.n_x)
    return n * evals / (e0.elapsed_time(e1) / 1e3)


ROWS = [("tiny", "auto"), ("mid", "auto"), ("precision", "dft"), ("precision", "split"),
        ("learned", "dft"), ("learned", "split"), ("differentiation", "auto"), ("mid", "sqnaf"),
        ("correlation", "auto"), ("correlation", "split")]


@pytest.mark.parametrize("which,path", ROWS)
def test_error_report(api, orc, which, path):
    """path "sqnaf": the matched-filter variant (h = x, no filter step) on the
    FFT path; its rate counts the hard-design score of each outer iteration."""
    w = getattr(wl, which)()
    matched = path == "sqnaf"
    p = {"auto": api.AF_PATH_AUTO, "sqnaf": api.AF_PATH_AUTO, "dft": api.AF_PATH_DFT,
         "split": api.AF_PATH_SPLIT_BF16}[path]
    chi_tol, db_tol = (1e-4, 0.1) if path == "split" else (1e-5, 0.05)
    x, h = _pair(orc, 77, w.M, w.N)
    if matched:
        h = x
    ctx = api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db, r_n=w.r_n, c=w.c,
                      n_h=0 if matched else w.n_h, n_x=w.n_x, lr_h=w.lr_h, lr_x=w.lr_x, path=p, matched=matched)
    xd, hd = torch.from_numpy(x).cuda(), torch.from_numpy(h).cuda()
    # |chi| on sampled cells (every cell of small grids)
    total = w.M * w.M * w.D * w.L
    cells = np.arange(total) if total <= 40000 else np.unique(
        (wl.uniform(78, 4000, 4) * total).astype(np.int64))
    chi = ctx.af_ambiguity(xd, hd).reshape(-1)     # the whole grid: 1.07 GB at the largest workload
    got = chi[torch.from_numpy(cells).cuda()].cpu().numpy()
    del chi
    ref = orc.ambiguity_cells(x, h, w.nu, w.k_lo, w.k_hi, cells)
    chi_err = np.max(np.abs(got - ref)) / w.N
    # loss terms, winning cell, gradient there
    gx = torch.empty((w.M, w.N), dtype=torch.complex64, device="cuda")
    gh = None if matched else torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(xd, hd, grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    cell = int(t[6 + int(t[5])])
    chi_c, ogx, ogh = orc.grad_at_cell(x, h, w.nu, w.k_lo, w.k_hi, cell, 1.0 / w.N, eps=w.eps,
                                       snrl_db=w.snrl_db)
    if matched:
        # h = x: the waveform's gradient is the sum of both partials
        og = ogx + ogh
        grad_err = np.max(np.abs(gx.cpu().numpy() - og)) / np.max(np.abs(og))
    else:
        scale = max(np.max(np.abs(ogx)), np.max(np.abs(ogh)))
        grad_err = max(np.max(np.abs(gx.cpu().numpy() - ogx)), np.max(np.abs(gh.cpu().numpy() - ogh))) / scale
    if which != "differentiation":
        r = orc.loss(x, h, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db)
        dpsl = max(abs(20 * np.log10(t[g] / r[k])) for g, k in ((2, "wapsl"), (3, "wcpsl")) if r[k] > 0)
    else:
        # max over 20,000 sampled cells cannot exceed the reported max; the reported
        # max is the oracle's |chi| at the reported cell
        dpsl = abs(20 * np.log10(t[1] / (abs(chi_c) / w.N)))
    eps_s = _evals_per_s(api, ctx, w, 5, matched)
    ctx.close()
    print(f"\n| {which} | {path} | {eps_s:,.0f} | {chi_err:.1e} | {dpsl:.4f} | {grad_err:.1e} |")
    assert chi_err <= chi_tol
    assert dpsl <= db_tol
    assert grad_err <= 1e-4
