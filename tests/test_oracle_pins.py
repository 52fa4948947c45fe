"""Pins for the FP64 oracle: checks against facts that do not come from the
oracle itself (library routines, closed forms, textbook sequences, invariants,
finite differences and the paper's worked example).  CPU only."""
import os

import numpy as np
import pytest

from paper_2604_25728_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = vals
    return out


def _random_pair(seed, M, N):
    x = wl.unit_phasors(seed, M, N)
    h = x + 0.3 * wl.complex_normal(seed, M, N)
    return x, h


# ------------------------------------------------------------------ Eq. 6 ----
def test_zero_doppler_row_is_numpy_correlation(orc):
    """At nu = 0, Eq. 6 is the aperiodic cross-correlation; numpy.correlate(a, v)
    returns c[k] = sum_n a[n+k] conj(v[n]) for lags -(len(v)-1)..len(a)-1."""
    M, N = 2, 23
    x, h = _random_pair(1, M, N)
    chi = orc.ambiguity(x, h, np.array([0.0]), -(N - 1), N - 1)
    for m in range(M):
        for l in range(M):
            ref = np.conj(np.correlate(h[l], x[m], mode="full"))
            np.testing.assert_allclose(chi[m, l, :, 0], ref, rtol=0, atol=1e-12)


def test_origin_cell_is_filter_inner_product(orc):
    """chi_mm(0, 0) = h_m^H x_m (Eq. 38) as numpy.vdot computes it."""
    M, N = 3, 31
    x, h = _random_pair(2, M, N)
    chi = orc.ambiguity(x, h, np.array([0.0, 0.25]), -3, 3)
    for m in range(M):
        assert abs(chi[m, m, 3, 0] - np.vdot(h[m], x[m])) < 1e-12


def test_full_grid_rows_match_numpy_ifft(orc):
    """On nu_j = -0.5 + j/L the Doppler sum of each delay row is an unnormalised
    inverse DFT of the sign-alternated lag products (numpy.fft.ifft)."""
    M, N, L = 2, 24, 32
    x, h = _random_pair(3, M, N)
    nu = wl.full_grid(L)
    chi = orc.ambiguity(x, h, nu, -(N - 1), N - 1)
    n = np.arange(N)
    for m in range(M):
        for l in range(M):
            for d, k in enumerate(range(-(N - 1), N)):
                hp = np.zeros(N, dtype=complex)
                valid = (n + k >= 0) & (n + k < N)
                hp[valid] = h[l][n[valid] + k]
                q = x[m] * np.conj(hp) * (-1.0) ** n
                ref = L * np.fft.ifft(q, L)
                np.testing.assert_allclose(chi[m, l, d], ref, rtol=0, atol=1e-10)


def test_parseval_on_full_grid(orc):
    """sum_j |chi(k, nu_j)|^2 = L sum_n |x(n)|^2 |h(n+k)|^2 for a full uniform
    grid with L >= N, for any grid offset."""
    M, N, L = 2, 20, 32
    x, h = _random_pair(4, M, N)
    nu = 0.137 + np.arange(L) / L
    chi = orc.ambiguity(x, h, nu, -(N - 1), N - 1)
    n = np.arange(N)
    for m in range(M):
        for l in range(M):
            for d, k in enumerate(range(-(N - 1), N)):
                valid = (n + k >= 0) & (n + k < N)
                rhs = L * np.sum(np.abs(x[m][valid]) ** 2 * np.abs(h[l][n[valid] + k]) ** 2)
                lhs = np.sum(np.abs(chi[m, l, d]) ** 2)
                assert abs(lhs - rhs) <= 1e-10 * max(1.0, rhs)


def test_dirichlet_kernel_zero_delay(orc):
    """h = x unimodular: |chi(0, nu)| = |sin(pi nu N) / sin(pi nu)|."""
    N = 40
    x = wl.unit_phasors(5, 1, N)
    nu = np.array([0.0013, 0.01, 0.1, 0.2371, -0.3, 0.49])
    chi = orc.ambiguity(x, x, nu, 0, 0)
    ref = np.abs(np.sin(np.pi * nu * N) / np.sin(np.pi * nu))
    np.testing.assert_allclose(np.abs(chi[0, 0, 0]), ref, rtol=1e-11, atol=1e-11)


def test_mirror_symmetry(orc):
    """|chi_{x,h}(k, nu)| = |chi_{h,x}(-k, -nu)|."""
    M, N = 2, 17
    x, h = _random_pair(6, M, N)
    nu = np.array([-0.31, -0.02, 0.0, 0.11, 0.4])
    a = orc.ambiguity(x, h, nu, -(N - 1), N - 1)
    b = orc.ambiguity(h, x, -nu, -(N - 1), N - 1)
    for m in range(M):
        for l in range(M):
            np.testing.assert_allclose(np.abs(a[m, l]), np.abs(b[l, m][::-1]), atol=1e-11)


def test_modulation_shifts_doppler_bin(orc):
    """x(n) -> x(n) e^{j 2 pi n / L} moves the response one bin up: chi'(k, nu_j)
    = chi(k, nu_{j+1}).  A sign error in the Doppler phasor fails this."""
    M, N, L = 1, 16, 16
    x, h = _random_pair(7, M, N)
    nu = wl.full_grid(L)
    a = orc.ambiguity(x, h, nu, -(N - 1), N - 1)
    xs = x * np.exp(2j * np.pi * np.arange(N) / L)
    b = orc.ambiguity(xs, h, nu, -(N - 1), N - 1)
    np.testing.assert_allclose(b[..., :-1], a[..., 1:], atol=1e-11)


def test_paper_index_origin_changes_no_magnitude(orc):
    """Eq. 6 counts n from 1; that is chi times e^{j 2 pi nu}, so every |chi|
    agrees with a sum taken over n = 1..N written with numpy.correlate after
    modulating x (the library computes the lag sum)."""
    N = 12
    x, h = _random_pair(8, 1, N)
    nu = 0.173
    n1 = np.arange(1, N + 1)
    chi = orc.ambiguity(x, h, np.array([nu]), -(N - 1), N - 1)[0, 0, :, 0]
    xm = x[0] * np.exp(2j * np.pi * n1 * nu)
    ref = np.conj(np.correlate(h[0], xm, mode="full"))
    np.testing.assert_allclose(np.abs(chi), np.abs(ref), atol=1e-12)
    np.testing.assert_allclose(chi * np.exp(2j * np.pi * nu), ref, atol=1e-12)


# ------------------------------------------------------------------ loss -----
def test_barker13_textbook_sidelobes(orc):
    """Matched Barker-13 at zero Doppler: max sidelobe 1 -> WAPSL = 1/13 with
    w = 1/N; SNRL term 0 at mu = 0 dB; PSLR -22.28 dB (Eq. 48)."""
    g = _read_golden("barker13.txt")
    code = np.array([float(v) for v in g["code"]]).reshape(1, -1).astype(complex)
    N = code.shape[1]
    r = orc.loss(code, code, np.array([0.0]), -(N - 1), N - 1, eps=0.1, snrl_db=0.0)
    assert abs(r["wapsl"] - float(g["max_sidelobe"][0]) / N) < 1e-14
    assert r["wcpsl"] == 0.0
    assert abs(r["snrl_term"]) < 1e-28
    assert abs(r["loss"] - 0.1 / N) < 1e-14
    met, snrl = orc.metrics(code, code, np.array([0.0]), -(N - 1), N - 1)
    assert abs(met[0] - float(g["pslr_db"][0])) < 1e-9
    assert abs(snrl[0]) < 1e-12


def test_auto_excludes_zero_delay_cross_includes_it(orc):
    """Two identical Barker channels: the cross term is the autocorrelation
    including its tau = 0 mainlobe (Eq. 9 keeps tau = 0), the auto term keeps
    only sidelobes (Eq. 8 drops tau = 0), and the WPSL is the larger (Eq. 7)."""
    code = np.array([float(v) for v in _read_golden("barker13.txt")["code"]])
    x = np.stack([code, code]).astype(complex)
    N = 13
    r = orc.loss(x, x, np.array([0.0]), -(N - 1), N - 1, eps=1.0, snrl_db=0.0)
    assert abs(r["wapsl"] - 1.0 / N) < 1e-14
    assert abs(r["wcpsl"] - 1.0) < 1e-14
    assert abs(r["wpsl"] - 1.0) < 1e-14 and r["cls"] == 1
    assert abs(r["loss"] - 1.0) < 1e-14
    D = 2 * N - 1
    m, l, d, j = np.unravel_index(r["cells"][1], (2, 2, D, 1))
    assert m != l and d - (N - 1) == 0


def test_snrl_identity_and_target(orc):
    """With ||x||^2 = ||h||^2 = N, SNRL (Eq. 10) = -20 log10 p_m (Eq. 38), and
    the penalty of Eq. 41 is the mean of (p_m - 10^(-mu/20))^2."""
    M, N = 3, 50
    x = wl.unit_phasors(9, M, N)
    h = orc.project(x + 0.5 * wl.complex_normal(9, M, N))
    r = orc.loss(x, h, np.array([0.0]), 0, 0, eps=0.3, snrl_db=0.7)
    _, snrl = orc.metrics(x, h, np.array([0.0]), 0, 0)
    p = np.abs(np.einsum("mn,mn->m", np.conj(h), x)) / N
    np.testing.assert_allclose(r["p"], p, rtol=1e-13)
    np.testing.assert_allclose(snrl, -20 * np.log10(p), rtol=1e-12)
    ptar = 10 ** (-0.7 / 20)
    assert abs(r["snrl_term"] - np.mean((p - ptar) ** 2)) < 1e-14
    assert abs(r["loss"] - (0.3 * r["wpsl"] + 0.7 * r["snrl_term"])) < 1e-14


def test_pnorm_tends_to_max(orc):
    """The p-norm variant of the class value tends to the exact max as p grows."""
    M, N = 2, 24
    x, h = _random_pair(10, M, N)
    nu = wl.full_grid(16)
    exact = orc.loss(x, h, nu, -(N - 1), N - 1)
    vals = [orc.loss(x, h, nu, -(N - 1), N - 1, pnorm=p)["wpsl"] for p in (8, 32, 256)]
    assert vals[0] > vals[1] > vals[2] > exact["wpsl"]
    assert vals[2] / exact["wpsl"] < 1.0 + 2.0 * np.log(2 * 47 * 16) / 256


# ------------------------------------------------------------------ gradient -
def _fd_check_xh(orc, x, h, nu, k_lo, k_hi, pnorm, eps, seed, ncoord=24, step=1e-6, tol=1e-6):
    terms, gx, gh = orc.grad_xh(x, h, nu, k_lo, k_hi, eps=eps, pnorm=pnorm)
    M, N = x.shape
    rng_idx = (wl.uniform(seed, ncoord, 3) * (M * N)).astype(int)
    which = (wl.uniform(seed, ncoord, 4) * 4).astype(int)
    for idx, wh in zip(rng_idx, which):
        m, n = divmod(int(idx), N)
        e = 1.0 if wh % 2 == 0 else 1j
        on_h = wh >= 2
        def f(s):
            xx, hh = x.copy(), h.copy()
            if on_h:
                hh[m, n] += s * e
            else:
                xx[m, n] += s * e
            return orc.loss(xx, hh, nu, k_lo, k_hi, eps=eps, pnorm=pnorm)["loss"]
        fd = (f(step) - f(-step)) / (2 * step)
        g = gh[m, n] if on_h else gx[m, n]
        an = g.real if e == 1.0 else g.imag
        assert abs(fd - an) <= tol * max(1.0, abs(an)), (m, n, wh, fd, an)


def test_gradient_exact_max_matches_finite_differences(orc):
    M, N = 2, 16
    x, h = _random_pair(11, M, N)
    _fd_check_xh(orc, x, h, wl.full_grid(16), -(N - 1), N - 1, 0.0, 0.1, seed=11)


def test_gradient_pnorm_matches_finite_differences(orc):
    M, N = 2, 12
    x, h = _random_pair(12, M, N)
    _fd_check_xh(orc, x, h, wl.full_grid(8), -5, 7, 8.0, 0.4, seed=12)


def test_gradient_invariances(orc):
    """A common phase rotation of any x_m or h_l leaves the loss unchanged, so
    sum_n Im(conj(x) grad x) = 0 and sum_n Re(conj(grad h) j h) = 0; the
    sidelobe term is 1-homogeneous in h and in x (Euler: Re<grad, v> = value)."""
    M, N = 3, 20
    x, h = _random_pair(13, M, N)
    nu = wl.full_grid(16)
    for eps, pn in ((0.1, 0.0), (0.5, 6.0)):
        t, gx, gh = orc.grad_xh(x, h, nu, -(N - 1), N - 1, eps=eps, pnorm=pn)
        for m in range(M):
            assert abs(np.sum(np.imag(np.conj(x[m]) * gx[m]))) < 1e-12
            assert abs(np.sum(np.real(np.conj(gh[m]) * 1j * h[m]))) < 1e-12
    for pn in (0.0, 6.0):
        t, gx, gh = orc.grad_xh(x, h, nu, -(N - 1), N - 1, eps=1.0, pnorm=pn)
        assert abs(np.sum(np.real(np.conj(gh) * h)) - t[1]) < 1e-12
        assert abs(np.sum(np.real(np.conj(gx) * x)) - t[1]) < 1e-12


def test_gradient_through_soft_quantizer_matches_finite_differences(orc):
    """dL/du through z = sigmoid(u), y = Q_A(z), x = e^{j 2 pi y}."""
    M, N, B, r_n = 2, 16, 4, 3
    rho, a = orc.thresholds(B, r_n)
    c = 40.0
    u = wl.logits(14, M, N, scale=1.5)
    h = orc.project(wl.unit_phasors(14, M, N) + 0.2 * wl.complex_normal(14, M, N))
    nu = wl.full_grid(16)
    kw = dict(nu=nu, k_lo=-(N - 1), k_hi=N - 1, eps=0.2, snrl_db=0.5)
    t, gu, gh = orc.loss_grad_u(u, h, rho, a, c, **kw)
    idx = (wl.uniform(14, 20, 5) * M * N).astype(int)
    for i in idx:
        m, n = divmod(int(i), N)
        step = 1e-6
        up, um = u.copy(), u.copy()
        up[m, n] += step
        um[m, n] -= step
        fp = orc.loss_grad_u(up, h, rho, a, c, **kw)[0][0]
        fm = orc.loss_grad_u(um, h, rho, a, c, **kw)[0][0]
        fd = (fp - fm) / (2 * step)
        assert abs(fd - gu[m, n]) <= 1e-5 * max(1.0, abs(gu[m, n])), (m, n, fd, gu[m, n])
    # the filter gradient of the soft chain is the plain filter gradient at x_soft
    xs, _ = orc.soft_waveform(u, rho, a, c)
    _, _, gh2 = orc.grad_xh(xs, h, nu, -(N - 1), N - 1, eps=0.2, snrl_db=0.5)
    np.testing.assert_allclose(gh, gh2, atol=1e-14)


# ------------------------------------------------------------------ quantizers
def test_worked_example_levels_eq25(orc):
    """B=4, r_n=3, c=300: the hard quantizer takes the 13 levels k/4, k=0..12
    (Eq. 25); the c -> infinity reading and the literal Eq. 43 agree there."""
    g = _read_golden("eq25_worked_example.txt")
    B, r_n, c = int(g["B"][0]), int(g["r_n"][0]), float(g["c"][0])
    levels = np.array([float(v) for v in g["levels"]])
    rho, a = orc.thresholds(B, r_n)
    z = np.linspace(0.0, 1.0, 4001)
    q, b = orc.hard_quantize(z, rho, B)
    np.testing.assert_array_equal(np.unique(q / B), levels)
    lit = orc.hard_quantize_literal(z, rho, a, c)
    np.testing.assert_allclose(lit, q / B, atol=1e-9)
    np.testing.assert_array_equal(b, q % B)
    assert set(np.unique(b)) == set(range(B))


def test_soft_quantizer_shape(orc):
    """Q_A is increasing, Q_A(0) ~ 0, Q_A(1) ~ r_n, the derivative matches
    finite differences, and large c gives the staircase q/B away from the
    thresholds."""
    B, r_n = 4, 3
    rho, a = orc.thresholds(B, r_n)
    z = np.linspace(0, 1, 997)
    y, dy = orc.soft_quantize(z, rho, a, 300.0)
    assert np.all(np.diff(y) > 0) and np.all(dy > 0)
    assert y[0] < 1e-9 and abs(y[-1] - r_n) < 1e-9
    s = 1e-7
    yp, _ = orc.soft_quantize(z + s, rho, a, 300.0)
    ym, _ = orc.soft_quantize(z - s, rho, a, 300.0)
    np.testing.assert_allclose((yp - ym) / (2 * s), dy, rtol=1e-5, atol=1e-6)
    zz = (np.arange(12) + 0.1) / 12 + 0.0
    yy, _ = orc.soft_quantize(zz, rho, a, 1e6)
    q, _ = orc.hard_quantize(zz, rho, B)
    np.testing.assert_allclose(yy, q / B, atol=1e-12)


def test_hard_quantizer_ties_count_as_reached(orc):
    """A value exactly on a threshold is counted (rho_i <= z)."""
    rho, _ = orc.thresholds(4, 2)
    q, _ = orc.hard_quantize(rho, rho, 4)
    np.testing.assert_array_equal(q, np.arange(1, rho.size + 1))


def test_init_logits_round_trip(orc):
    """The initial logits map back to the drawn phase indices."""
    B, r_n = 16, 100
    rho, _ = orc.thresholds(B, r_n)
    b = wl.phase_indices(3, 2, 64, B)
    u = orc.init_logits(b, B, r_n)
    q, x = orc.hard_waveform(u, rho, B)
    np.testing.assert_array_equal(q % B, b)
    np.testing.assert_allclose(x, np.exp(2j * np.pi * b / B), atol=1e-14)


# ------------------------------------------------------------------ projection, Adam
def test_projection_energy(orc):
    M, N = 4, 33
    h = 3.0 * wl.complex_normal(15, M, N)
    hp = orc.project(h)
    np.testing.assert_allclose(np.sum(np.abs(hp) ** 2, axis=1), N, rtol=1e-13)
    for m in range(M):
        ratio = hp[m] / h[m]
        assert np.allclose(ratio, ratio[0], rtol=1e-13) and ratio[0].real > 0


def test_adam_matches_torch():
    """The oracle's Adam equals torch.optim.Adam (same hyper-parameters)."""
    torch = pytest.importorskip("torch")
    import oracle as orc
    n = 37
    theta = wl.normal(16, n, 1)
    p = torch.nn.Parameter(torch.tensor(theta.copy(), dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=0.05, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(n)
    v = np.zeros(n)
    th = theta.copy()
    for t in range(1, 6):
        g = wl.normal(16, n, 10 + t)
        orc.adam(th, g, m, v, t, 0.05)
        opt.zero_grad()
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------ Algorithm 1
def test_outer_iteration_structure(orc):
    """One outer iteration: Step A leaves u alone and keeps ||h_m||^2 = N;
    Step B leaves h alone; the first loss is that of (X_hard(u), H)."""
    w = wl.small(2, 16, 4, 16, r_n=5)
    rho, a = orc.thresholds(w.B, w.r_n)
    b = wl.phase_indices(1, w.M, w.N, w.B)
    u = orc.init_logits(b, w.B, w.r_n)
    x0 = np.exp(2j * np.pi * b / w.B)
    h = orc.project(x0 + 0.1 * wl.complex_normal(1, w.M, w.N))
    st = dict(u=u.copy(), h=h.copy(), mu=np.zeros_like(u), vu=np.zeros_like(u),
              mh=np.zeros_like(h), vh=np.zeros_like(h), t_x=0, t_h=0)
    cfg = dict(nu=w.nu, k_lo=w.k_lo, k_hi=w.k_hi, eps=w.eps, snrl_db=w.snrl_db, B=w.B,
               rho=rho, a=a, c=w.c, n_h=3, n_x=0, lr_h=w.lr_h, lr_x=w.lr_x)
    losses, _ = orc.sqngd_outer(st, cfg)
    first = orc.loss(x0, h, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db)["loss"]
    assert abs(losses[0] - first) < 1e-14
    np.testing.assert_array_equal(st["u"], u)
    np.testing.assert_allclose(np.sum(np.abs(st["h"]) ** 2, axis=1), w.N, rtol=1e-12)
    assert st["t_h"] == 3 and st["t_x"] == 0
    h_after = st["h"].copy()
    cfg.update(n_h=0, n_x=2)
    orc.sqngd_outer(st, cfg)
    np.testing.assert_array_equal(st["h"], h_after)
    assert st["t_x"] == 2 and not np.array_equal(st["u"], u)


def test_grad_at_cell_equals_full_gradient_at_that_cell(orc):
    """The no-scan gradient equals the full-scan gradient differentiated at the
    same cell (the argmax, and a non-argmax cell passed explicitly)."""
    M, N = 2, 14
    x, h = _random_pair(17, M, N)
    nu = wl.full_grid(8)
    r = orc.loss(x, h, nu, -(N - 1), N - 1, eps=0.3, snrl_db=0.4)
    for cell in (r["cells"][r["cls"]], 37):
        _, gx, gh = orc.grad_xh(x, h, nu, -(N - 1), N - 1, eps=0.3, snrl_db=0.4, use_cell=cell)
        chi, gx2, gh2 = orc.grad_at_cell(x, h, nu, -(N - 1), N - 1, cell, 1.0 / N, eps=0.3, snrl_db=0.4)
        np.testing.assert_allclose(gx2, gx, atol=1e-14)
        np.testing.assert_allclose(gh2, gh, atol=1e-14)
        full = orc.ambiguity(x, h, nu, -(N - 1), N - 1).reshape(-1)
        assert abs(chi - full[cell]) < 1e-12


# ------------------------------------------------------------------ SQNAF (h = x)
def test_matched_gradient_matches_finite_differences(orc):
    """SQNAF takes every filter equal to its waveform: the gradient of
    L(x, x) against central differences of the loss with both arguments
    moved together.  Non-unimodular x so that the SNRL term also contributes;
    a one-sided delay window and an offset grid so the max is unique."""
    M, N = 2, 10
    x = wl.unit_phasors(21, M, N) + 0.4 * wl.complex_normal(21, M, N)
    nu = 0.0137 + np.arange(8) / 8
    k_lo, k_hi = 1, 6
    for eps in (0.1, 0.7):
        _, g = orc.grad_matched(x, nu, k_lo, k_hi, eps=eps, snrl_db=0.5)
        idx = (wl.uniform(22, 16, 3) * (M * N)).astype(int)
        for t, i in enumerate(idx):
            m, n = divmod(int(i), N)
            e = 1.0 if t % 2 == 0 else 1j
            def f(s):
                xx = x.copy()
                xx[m, n] += s * e
                return orc.loss(xx, xx, nu, k_lo, k_hi, eps=eps, snrl_db=0.5)["loss"]
            fd = (f(1e-6) - f(-1e-6)) / 2e-6
            an = g[m, n].real if e == 1.0 else g[m, n].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (eps, m, n, fd, an)


def test_matched_gradient_is_sum_of_partials_and_not_either_alone(orc):
    """The matched gradient is neither partial alone: with h = x both the
    transmit and the filter side move."""
    M, N = 2, 12
    x = wl.unit_phasors(23, M, N)
    nu = 0.021 + np.arange(8) / 8
    _, g = orc.grad_matched(x, nu, 1, 9, eps=0.3)
    _, gx, gh = orc.grad_xh(x, x, nu, 1, 9, eps=0.3)
    np.testing.assert_allclose(g, gx + gh, atol=1e-15)
    assert np.max(np.abs(gh)) > 0.1 * np.max(np.abs(g)) and np.max(np.abs(gx)) > 0.1 * np.max(np.abs(g))


def test_matched_snrl_term_has_no_phase_gradient(orc):
    """With h = x a unimodular waveform has p_m = 1 whatever its phases, so
    the SNRL term (eps = 0) is constant along the transmit chain: dL/du = 0."""
    M, N, B, r_n = 2, 16, 4, 3
    rho, a = orc.thresholds(B, r_n)
    u = wl.logits(24, M, N, scale=1.5)
    t, gu = orc.loss_grad_u_matched(u, rho, a, 40.0, wl.full_grid(16), -(N - 1), N - 1, eps=0.0,
                                    snrl_db=1.0)
    ptar = 10 ** (-1.0 / 20)
    assert abs(t[4] - (1 - ptar) ** 2) < 1e-12
    assert np.max(np.abs(gu)) < 1e-12


def test_matched_soft_chain_matches_finite_differences(orc):
    M, N, B, r_n = 2, 12, 4, 3
    rho, a = orc.thresholds(B, r_n)
    c = 40.0
    u = wl.logits(25, M, N, scale=1.5)
    kw = dict(nu=0.011 + np.arange(8) / 8, k_lo=1, k_hi=8, eps=0.3, snrl_db=0.5)
    _, gu = orc.loss_grad_u_matched(u, rho, a, c, **kw)
    for i in (wl.uniform(25, 12, 5) * M * N).astype(int):
        m, n = divmod(int(i), N)
        up, um = u.copy(), u.copy()
        up[m, n] += 1e-6
        um[m, n] -= 1e-6
        fd = (orc.loss_grad_u_matched(up, rho, a, c, **kw)[0][0]
              - orc.loss_grad_u_matched(um, rho, a, c, **kw)[0][0]) / 2e-6
        assert abs(fd - gu[m, n]) <= 1e-5 * max(1.0, abs(gu[m, n])), (m, n, fd, gu[m, n])
    # the loss is that of the soft waveform used as its own filter
    xs, _ = orc.soft_waveform(u, rho, a, c)
    r = orc.loss(xs, xs, **kw)
    assert abs(orc.loss_grad_u_matched(u, rho, a, c, **kw)[0][0] - r["loss"]) < 1e-14


def test_sqnaf_outer_iteration_structure(orc):
    """SQNAF outer iteration: the first value scores (X_hard, X_hard); one
    transmit step is Adam on u with the matched soft-chain gradient."""
    w = wl.small(2, 16, 4, 16, r_n=5)
    rho, a = orc.thresholds(w.B, w.r_n)
    b = wl.phase_indices(2, w.M, w.N, w.B)
    u = orc.init_logits(b, w.B, w.r_n)
    st = dict(u=u.copy(), mu=np.zeros_like(u), vu=np.zeros_like(u), t_x=0)
    cfg = dict(nu=w.nu, k_lo=w.k_lo, k_hi=w.k_hi, eps=w.eps, snrl_db=w.snrl_db, B=w.B,
               rho=rho, a=a, c=w.c, n_x=1, lr_x=1e-2)
    losses, wpsl = orc.sqnaf_outer(st, cfg)
    x0 = np.exp(2j * np.pi * b / w.B)
    r0 = orc.loss(x0, x0, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db)
    assert abs(losses[0] - r0["loss"]) < 1e-14 and abs(wpsl[0] - r0["wpsl"]) < 1e-14
    t1, gu = orc.loss_grad_u_matched(u, rho, a, w.c, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db)
    assert abs(losses[1] - t1[0]) < 1e-14
    theta, m, v = u.copy(), np.zeros_like(u), np.zeros_like(u)
    orc.adam(theta, gu, m, v, 1, 1e-2)
    np.testing.assert_array_equal(st["u"], theta)
    assert st["t_x"] == 1


# ------------------------------------------------------------------ trainable thresholds
def test_threshold_gradient_matches_finite_differences(orc):
    """dL/drho_i through y = Q_A(z; rho) (Eq. 24) against central differences
    of the loss with rho_i moved, at thresholds inside the elements' windows."""
    M, N, B, r_n, c = 2, 12, 4, 3, 40.0
    rho, a = orc.thresholds(B, r_n)
    u = wl.logits(31, M, N, scale=1.5)
    h = orc.project(wl.unit_phasors(31, M, N) + 0.2 * wl.complex_normal(31, M, N))
    kw = dict(nu=wl.full_grid(16), k_lo=-(N - 1), k_hi=N - 1, eps=0.3, snrl_db=0.5)
    _, gu, gr = orc.loss_grad_u_rho(u, h, rho, a, c, **kw)
    _, gu2, _ = orc.loss_grad_u(u, h, rho, a, c, **kw)
    np.testing.assert_allclose(gu, gu2, atol=1e-14)
    order = np.argsort(-np.abs(gr))
    assert np.abs(gr[order[0]]) > 1e-3
    for i in list(order[:6]) + [int(order[-1])]:
        rp, rm = rho.copy(), rho.copy()
        rp[i] += 1e-7
        rm[i] -= 1e-7
        fd = (orc.loss_grad_u_rho(u, h, rp, a, c, **kw)[0][0] - orc.loss_grad_u_rho(u, h, rm, a, c, **kw)[0][0]) / 2e-7
        assert abs(fd - gr[i]) <= 1e-5 * max(1.0, abs(gr[i])), (i, fd, gr[i])


def test_threshold_projection_is_the_euclidean_projection():
    """Against a generic constrained least-squares solver on small random sets:
    the nearest 0 <= rho_0 <= ... <= rho_{K-1} <= 1."""
    import importlib
    orc = importlib.import_module("oracle")
    opt = pytest.importorskip("scipy.optimize")
    for seed in range(12):
        K = 3 + seed % 6
        r = wl.uniform(40 + seed, K, 2) * 1.4 - 0.2          # some outside [0, 1], unordered
        got = orc.project_thresholds(r)
        cons = [{"type": "ineq", "fun": (lambda x, i=i: x[i + 1] - x[i])} for i in range(K - 1)]
        res = opt.minimize(lambda x: np.sum((x - r) ** 2), np.clip(np.sort(r), 0, 1), method="SLSQP",
                           bounds=[(0.0, 1.0)] * K, constraints=cons, options={"ftol": 1e-14, "maxiter": 500})
        assert np.all(np.diff(got) >= 0) and got.min() >= 0 and got.max() <= 1
        assert np.sum((got - r) ** 2) <= res.fun + 1e-9, (seed, got, res.x)
        np.testing.assert_allclose(got, res.x, atol=1e-5)


def test_threshold_projection_keeps_ordered_sets_and_pools_means(orc):
    rho, _ = orc.thresholds(4, 5)
    np.testing.assert_array_equal(orc.project_thresholds(rho), rho)
    r = np.array([0.1, 0.5, 0.3, 0.4, 0.9, 0.8])
    got = orc.project_thresholds(r)
    # pooled blocks {0.5, 0.3, 0.4} -> 0.4 and {0.9, 0.8} -> 0.85, means preserved
    np.testing.assert_allclose(got, [0.1, 0.4, 0.4, 0.4, 0.85, 0.85], atol=1e-15)


def test_outer_iteration_with_frozen_thresholds_equals_plain(orc):
    """lr_rho = 0 leaves rho untouched and reproduces the plain outer iteration;
    lr_rho > 0 moves rho and keeps it ordered inside [0, 1]."""
    w = wl.small(2, 16, 4, 16, r_n=5)
    rho, a = orc.thresholds(w.B, w.r_n)
    b = wl.phase_indices(3, w.M, w.N, w.B)
    u = orc.init_logits(b, w.B, w.r_n)
    h = orc.project(np.exp(2j * np.pi * b / w.B) + 0.1 * wl.complex_normal(3, w.M, w.N))
    cfg = dict(nu=w.nu, k_lo=w.k_lo, k_hi=w.k_hi, eps=w.eps, snrl_db=w.snrl_db, B=w.B, rho=rho, a=a,
               c=40.0, n_h=2, n_x=3, lr_h=w.lr_h, lr_x=1e-2, lr_rho=0.0)
    z = lambda: dict(u=u.copy(), h=h.copy(), mu=np.zeros_like(u), vu=np.zeros_like(u), mh=np.zeros_like(h),
                     vh=np.zeros_like(h), rho=rho.copy(), mr=np.zeros_like(rho), vr=np.zeros_like(rho),
                     t_x=0, t_h=0)
    s1, s2 = z(), z()
    l1, _ = orc.sqngd_outer_rho(s1, cfg)
    l2, _ = orc.sqngd_outer(s2, cfg)
    np.testing.assert_array_equal(l1, l2)
    np.testing.assert_array_equal(s1["u"], s2["u"])
    np.testing.assert_array_equal(s1["rho"], rho)
    cfg["lr_rho"] = 1e-3
    s3 = z()
    orc.sqngd_outer_rho(s3, cfg)
    assert not np.array_equal(s3["rho"], rho)
    assert np.all(np.diff(s3["rho"]) >= 0) and s3["rho"].min() >= 0 and s3["rho"].max() <= 1


def test_weighted_classes_by_enumeration(orc):
    """WAPSL/WCPSL with a non-square [D][L] weight map (D != L), against the
    pinned ambiguity and the class definitions of Eqs. 8-9 applied by
    enumeration: every cell of positive weight, auto without tau = 0."""
    M, N, L = 2, 11, 8
    k_lo, k_hi = -6, 8
    D = k_hi - k_lo + 1
    x, h = _random_pair(41, M, N)
    nu = 0.013 + np.arange(L) / L
    w = wl.uniform(42, D * L, 1).reshape(D, L)
    w[w < 0.2] = 0.0
    chi = np.abs(orc.ambiguity(x, h, nu, k_lo, k_hi))
    best = [0.0, 0.0]
    for m in range(M):
        for l in range(M):
            for d in range(D):
                if m == l and k_lo + d == 0:
                    continue
                for j in range(L):
                    if w[d, j] > 0:
                        c = 0 if m == l else 1
                        best[c] = max(best[c], w[d, j] * chi[m, l, d, j])
    r = orc.loss(x, h, nu, k_lo, k_hi, weights=w, eps=0.4, snrl_db=0.5)
    assert abs(r["wapsl"] - best[0]) < 1e-12 and abs(r["wcpsl"] - best[1]) < 1e-12
    assert abs(r["wpsl"] - max(best)) < 1e-12


def test_acceptance_metrics_by_enumeration(orc):
    """Eq. 48 over the ROI (cells of positive weight; auto without tau = 0) and
    the SNRL of Eq. 10, against the pinned ambiguity by enumeration."""
    M, N, L = 2, 13, 8
    k_lo, k_hi = -5, 9
    D = k_hi - k_lo + 1
    x, h = _random_pair(43, M, N)
    h = orc.project(h)
    nu = 0.021 + np.arange(L) / L
    w = wl.uniform(44, D * L, 1).reshape(D, L)
    w[w < 0.35] = 0.0
    chi = np.abs(orc.ambiguity(x, h, nu, k_lo, k_hi))
    psl = [0.0, 0.0]
    for m in range(M):
        for l in range(M):
            for d in range(D):
                if m == l and k_lo + d == 0:
                    continue
                for j in range(L):
                    if w[d, j] > 0:
                        c = 0 if m == l else 1
                        psl[c] = max(psl[c], chi[m, l, d, j])
    out, snrl = orc.metrics(x, h, nu, k_lo, k_hi, weights=w)
    np.testing.assert_allclose(out[:2], 20 * np.log10(np.array(psl) / N), atol=1e-12)
    assert abs(out[2] - max(out[0], out[1])) < 1e-12
    p = np.abs(np.sum(x * np.conj(h), axis=1)) / N
    np.testing.assert_allclose(snrl, -20 * np.log10(p), atol=1e-12)
    assert abs(out[3] - np.max(snrl)) < 1e-12


# ------------------------------------------------ sampled cells, rank-one FD ----
def test_ambiguity_cells_decode_on_a_non_square_grid(orc):
    """The sampled-cell evaluator (the checker of every full-size GPU test)
    decodes ((m M + l) D + d) L + j like the full grid: random cells of a grid
    with D != L, a delay window that is not centred, an offset Doppler grid
    and M = 3 (so a swapped m/l, d/j or D/L decode lands on another cell)."""
    M, N, L, k_lo, k_hi = 3, 37, 11, -20, 8
    nu = wl.full_grid(L) + 0.013
    x, h = _random_pair(21, M, N)
    ref = orc.ambiguity(x, h, nu, k_lo, k_hi).reshape(-1)
    D = k_hi - k_lo + 1
    assert D != L
    cells = np.unique(np.concatenate([(wl.uniform(22, 400) * ref.size).astype(np.int64),
                                      [0, ref.size - 1, L - 1, L, D * L - 1, D * L, M * D * L + 5]]))
    got = orc.ambiguity_cells(x, h, nu, k_lo, k_hi, cells)
    np.testing.assert_allclose(got, ref[cells], rtol=0, atol=1e-12)


def _replaced(a, r, c, v):
    b = a.copy()
    b[r, c] = v
    return b


@pytest.mark.parametrize("pnorm", [0.0, 8.0])
def test_fd_losses_equal_full_reevaluation(orc, pnorm):
    """The rank-one finite-difference losses equal the loss re-evaluated in
    full on explicitly perturbed inputs (x and h samples, both sides, samples
    at the ends of a row, a non-centred delay window, a weight map and the
    p-norm variant)."""
    M, N, L, k_lo, k_hi = 3, 20, 16, -15, 9
    nu = wl.full_grid(L) + 0.02
    x, h = _random_pair(31, M, N)
    D = k_hi - k_lo + 1
    weights = 0.05 * (1.0 + wl.uniform(32, D * L).reshape(D, L))
    weights[3, :4] = 0.0
    coords = []
    for i, (t, r, c) in enumerate([(0, 0, 0), (0, 2, 19), (1, 1, 7), (1, 0, 19), (0, 1, 10), (1, 2, 0)]):
        base = (x if t == 0 else h)[r, c]
        dv = 1e-3 * np.exp(1j * (0.7 + i))
        coords.append((t, r, c, base + dv, base - dv))
    for w in (None, weights):
        lp, lm = orc.fd_losses(x, h, nu, k_lo, k_hi, coords, weights=w, eps=0.3, snrl_db=0.7, pnorm=pnorm)
        for i, (t, r, c, vp, vm) in enumerate(coords):
            for v, got in ((vp, lp[i]), (vm, lm[i])):
                xx = _replaced(x, r, c, v) if t == 0 else x
                hh = _replaced(h, r, c, v) if t == 1 else h
                ref = orc.loss(xx, hh, nu, k_lo, k_hi, weights=w, eps=0.3, snrl_db=0.7, pnorm=pnorm)["loss"]
                assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (i, got, ref)


def test_fd_losses_give_the_analytic_gradient(orc):
    """Central differences of the rank-one losses reproduce the oracle's
    analytic gradient (dL/dRe + j dL/dIm) at real and imaginary steps."""
    M, N, L = 2, 24, 32
    nu = wl.full_grid(L)
    x, h = _random_pair(33, M, N)
    _, gx, gh = orc.grad_xh(x, h, nu, -(N - 1), N - 1, eps=0.2, snrl_db=0.4, pnorm=6.0)
    st = 1e-5
    coords = []
    picks = [(0, 0, 3), (0, 1, 17), (1, 0, 5), (1, 1, 23)]
    for t, r, c in picks:
        base = (x if t == 0 else h)[r, c]
        coords += [(t, r, c, base + st, base - st), (t, r, c, base + 1j * st, base - 1j * st)]
    lp, lm = orc.fd_losses(x, h, nu, -(N - 1), N - 1, coords, eps=0.2, snrl_db=0.4, pnorm=6.0)
    fd = (lp - lm) / (2 * st)
    for i, (t, r, c) in enumerate(picks):
        g = (gx if t == 0 else gh)[r, c]
        assert abs(fd[2 * i] - g.real) <= 1e-6 * np.abs(gx).max()
        assert abs(fd[2 * i + 1] - g.imag) <= 1e-6 * np.abs(gx).max()


# ------------------------------------------------------------- stopping rule ----
def test_stop_rule_by_hand():
    """Algorithm 1's stopping test on hand-made WPSL sequences: strict
    improvement resets the count, equal values do not, the patience-th
    iteration without improvement is the last one, T bounds the run, and a
    resumed record continues the count."""
    import oracle as orc
    # best at t = 3 (3 < 4); t = 4, 5 bring nothing: stop after t = 5
    assert orc.stop_rule([5, 4, 4, 3, 3, 3, 3, 1], 2, 100) == (6, 1, 3, 3)
    # the first iteration always improves on a fresh record
    assert orc.stop_rule([7.0] * 10, 3, 100) == (4, 1, 7.0, 0)
    # T reached first
    assert orc.stop_rule([9, 8, 7, 6, 5], 3, 4) == (4, 2, 6, 3)
    # resumed at t0 = 10 with the best at iteration 8: the count continues (stop after t = 11)
    assert orc.stop_rule([2.0, 2.0, 2.0], 3, 100, best_wpsl=1.5, best_outer=8, t0=10) == (2, 1, 1.5, 8)
    # NaN never improves: a fresh record stops after `patience` iterations
    assert orc.stop_rule([float("nan")] * 5, 2, 100)[:2] == (2, 1)
