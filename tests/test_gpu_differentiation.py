"""The differentiation workload's checks (M=4, N=2048, B=64, every delay,
2048 bins): the library gradient behind api.AfLoss (a torch.autograd
Function) against central finite differences of the FP64 oracle's loss, for
the paper's exact max and for the p-norm loss with its dense adjoint; and the
dense adjoint element by element at the large-transform launch shapes with
no override of the radix.

Finite differences: step 1e-4 on 64 seeded coordinates -- 32 transmit
logits u_m(n) (through the soft chain z = sigmoid(u), Eq. 24, x = e^{j 2 pi
y}) and 32 filter taps (16 real, 16 imaginary parts).  The oracle evaluates
each perturbed loss by a rank-one update of chi (only the pairs of the
perturbed row move), checked against full re-evaluation on CPU.  Bar: every
coordinate within 2e-3 of the largest checked gradient (FP32 against FP64:
the FP64 differences carry a truncation error of order step^2 and the FP32
soft quantizer a relative error near 1e-5).
"""
import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STEP = 1e-4
FD_TOL = 2e-3


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import api as a
    return a


def _coords(seed, M, N, n_u=32, n_h=32):
    """Seeded distinct coordinates: (kind, row, col) with kind 'u', 'hr', 'hi'."""
    r = wl.uniform(seed, 4 * (n_u + n_h), 3)
    out, seen = [], set()
    i = 0
    while len(out) < n_u + n_h:
        kind = "u" if len(out) < n_u else ("hr" if len(out) < n_u + n_h // 2 else "hi")
        m, n = int(r[i] * M), int(r[i + 1] * N)
        i += 2
        if (kind, m, n) in seen:
            continue
        seen.add((kind, m, n))
        out.append((kind, m, n))
    return out


def _fd_gradient(orc, w, u, h, coords, pnorm):
    """Central differences of the FP64 loss at the FP32 inputs u (logits) and
    h (filters): logit coordinates move one sample of the soft waveform.
    Returns (differences, the loss at the unperturbed inputs)."""
    rho, a = orc.thresholds(w.B, w.r_n)
    rho32 = rho.astype(np.float32).astype(np.float64)
    u64 = u.astype(np.float64)
    x, _ = orc.soft_waveform(u64, rho32, a, w.c)
    h64 = h.astype(np.complex128)
    oc = []
    for kind, m, n in coords:
        if kind == "u":
            up, um = u64.copy(), u64.copy()
            up[m, n] += STEP
            um[m, n] -= STEP
            xp = orc.soft_waveform(up[m:m + 1, n:n + 1], rho32, a, w.c)[0][0, 0]
            xm = orc.soft_waveform(um[m:m + 1, n:n + 1], rho32, a, w.c)[0][0, 0]
            oc.append((0, m, n, xp, xm))
        else:
            d = STEP if kind == "hr" else 1j * STEP
            oc.append((1, m, n, h64[m, n] + d, h64[m, n] - d))
    oc.append((1, 0, 0, h64[0, 0], h64[0, 0]))          # no change: the loss itself
    lp, lm = orc.fd_losses(x, h64, w.nu, w.k_lo, w.k_hi, oc, eps=w.eps, snrl_db=w.snrl_db, pnorm=pnorm)
    return (lp[:-1] - lm[:-1]) / (2 * STEP), lp[-1]


@pytest.mark.parametrize("pnorm", [0.0, 8.0])
def test_autograd_gradient_matches_finite_differences_at_full_size(api, orc, pnorm):
    w = wl.differentiation()
    u = (1.5 * wl.logits(51, w.M, w.N)).astype(np.float32)
    x0 = np.exp(2j * np.pi * wl.phase_indices(51, w.M, w.N, w.B) / w.B)
    h = orc.project(x0 + 0.3 * wl.complex_normal(51, w.M, w.N)).astype(np.complex64)
    ctx = api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db, r_n=w.r_n, c=w.c,
                      pnorm=pnorm)
    ut = torch.from_numpy(u).cuda().requires_grad_(True)
    ht = torch.from_numpy(h).cuda().requires_grad_(True)
    loss = api.AfLoss.apply(ut, ht, ctx)
    loss.backward()
    ctx.af_sync()
    gu, gh = ut.grad.cpu().numpy(), ht.grad.cpu().numpy()
    coords = _coords(52, w.M, w.N)
    fd, ref = _fd_gradient(orc, w, u, h, coords, pnorm)
    lib = np.array([gu[m, n] if k == "u" else (gh[m, n].real if k == "hr" else gh[m, n].imag)
                    for k, m, n in coords])
    scale = np.max(np.abs(fd))
    assert scale > 0
    err = np.abs(lib - fd)
    assert np.max(err) <= FD_TOL * scale, (np.max(err) / scale, coords[int(np.argmax(err))])
    # the loss the forward pass returned is the FP64 loss at the same inputs
    assert abs(float(loss.detach().cpu()) - ref) <= 1e-4 * abs(ref)
    ctx.close()


@pytest.mark.parametrize("pn", [7.0, 8.0, 16.0])
@pytest.mark.parametrize("L", [1024, 2048])
def test_dense_adjoint_at_large_transforms_default_radix(api, orc, L, pn):
    """The p-norm loss and its dense adjoint, element by element, at the
    transform lengths of the differentiation workload's launch shapes with
    the library's own choice of radix and CTA width (no override), every
    delay; p = 7 takes the general power, even p the multiplication-only one."""
    M, N = 3, 600
    nu = wl.full_grid(L)
    x = wl.unit_phasors(600 + L, M, N).astype(np.complex64)
    h = orc.project(x.astype(np.complex128) + 0.3 * wl.complex_normal(600 + L, M, N)).astype(np.complex64)
    ctx = api.Context(M, N, 4, nu, -(N - 1), N - 1, r_n=100, eps=0.3, snrl_db=0.5, pnorm=pn)
    gx = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(gx)
    terms, _, _ = ctx.af_loss_grad_xh(torch.from_numpy(x).cuda(), torch.from_numpy(h).cuda(), grad_x=gx, grad_h=gh)
    ctx.af_sync()
    t = terms.cpu().numpy()
    ot, ogx, ogh = orc.grad_xh(x, h, nu, -(N - 1), N - 1, eps=0.3, snrl_db=0.5, pnorm=pn)
    np.testing.assert_allclose(t[[0, 2, 3, 4]], ot[[0, 2, 3, 4]], rtol=2e-5, atol=1e-6)
    assert int(t[5]) == int(ot[5])
    scale = max(np.max(np.abs(ogx)), np.max(np.abs(ogh)))
    assert np.max(np.abs(gx.cpu().numpy() - ogx)) <= 2e-4 * scale
    assert np.max(np.abs(gh.cpu().numpy() - ogh)) <= 2e-4 * scale
    ctx.close()


def test_forward_pass_alone_skips_the_adjoint(api, orc):
    """With no gradient output the p-norm loss runs no dense adjoint: the
    terms equal those of the full evaluation."""
    M, N, L = 2, 100, 128
    nu = wl.full_grid(L)
    x = wl.unit_phasors(77, M, N).astype(np.complex64)
    h = orc.project(x.astype(np.complex128) + 0.3 * wl.complex_normal(77, M, N)).astype(np.complex64)
    ctx = api.Context(M, N, 4, nu, -(N - 1), N - 1, r_n=10, pnorm=8.0)
    xd, hd = torch.from_numpy(x).cuda(), torch.from_numpy(h).cuda()
    gx = torch.empty_like(xd)
    gh = torch.empty_like(xd)
    full, _, _ = ctx.af_loss_grad_xh(xd, hd, grad_x=gx, grad_h=gh)
    alone, _, _ = ctx.af_loss_grad_xh(xd, hd)
    ctx.af_sync()
    assert torch.equal(full, alone)
    ctx.close()
