"""The oracle's pins catch plausible mistakes: each case plants one mistake
(a flipped sign or conjugate, a dropped term, a swapped index, a wrong
constant or comparison) in a scratch copy of oracle/sqngd_oracle.c, builds
it, and runs the pin suite against it; the suite must fail.  CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sqngd_oracle.c")

MUTATIONS = [
    # (name, exact text, replacement)
    ("phasor sign of Eq. 6", "return cos(TWO_PI * f) + I * sin(TWO_PI * f);",
     "return cos(TWO_PI * f) - I * sin(TWO_PI * f);"),
    ("conjugate on the waveform instead of the filter", "s += xm[n] * conj(hl[p]) * phasor",
     "s += conj(xm[n]) * hl[p] * phasor"),
    ("auto class keeps tau = 0", "if (m == l) return (k == 0) ? -1 : 0;", "if (m == l) return 0;"),
    ("SNRL coefficient without (1 - eps)", "cplx G = (1.0 - eps) * (2.0 / M) * (p[m] - ptar)",
     "cplx G = (2.0 / M) * (p[m] - ptar)"),
    ("SNRL coefficient at a given cell without (1 - eps)", "cplx G = (1.0 - eps) * (2.0 / M) * (am / N - ptar)",
     "cplx G = (2.0 / M) * (am / N - ptar)"),
    ("quantizer scale a = 1/B", "if (a) *a = 1.0 / (2.0 * B);", "if (a) *a = 1.0 / B;"),
    ("filter gradient without conj(G)", "gh[(size_t)l * N + p] += conj(G) * x[(size_t)m * N + n] * e;",
     "gh[(size_t)l * N + p] += G * x[(size_t)m * N + n] * e;"),
    ("chain rule takes Re instead of Im",
     "double gy = TWO_PI * cimag(conj(xc[e]) * gxc[e]);\n        double z = 1.0 / (1.0 + exp(-u[e]));\n        gu[e] =",
     "double gy = TWO_PI * creal(conj(xc[e]) * gxc[e]);\n        double z = 1.0 / (1.0 + exp(-u[e]));\n        gu[e] ="),
    ("threshold chain takes Re instead of Im",
     "double gy = TWO_PI * cimag(conj(xc[e]) * gxc[e]);\n        double z = 1.0 / (1.0 + exp(-u[e]));\n        if (gu)",
     "double gy = TWO_PI * creal(conj(xc[e]) * gxc[e]);\n        double z = 1.0 / (1.0 + exp(-u[e]));\n        if (gu)"),
    ("matched chain takes Re instead of Im", "double gy = TWO_PI * cimag(conj(xc[e]) * gc[e]);",
     "double gy = TWO_PI * creal(conj(xc[e]) * gc[e]);"),
    ("hard quantizer counts rho < z", "if (rho[i] <= z[e]) ++cnt;", "if (rho[i] < z[e]) ++cnt;"),
    ("weight map indexed [L][D]", "return c->w ? c->w[(size_t)d * c->L + j] : 1.0 / (double)c->N;",
     "return c->w ? c->w[(size_t)j * (c->k_hi - c->k_lo + 1) + d] : 1.0 / (double)c->N;"),
    ("Adam without bias correction", "double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);",
     "double c1 = 1.0, c2 = 1.0;"),
    ("projection scales by N/e", "double s = sqrt((double)N / e);", "double s = (double)N / e;"),
    ("pooled mean divides by the last block", "val[nb - 2] = tot / cnt[nb - 2];", "val[nb - 2] = tot / cnt[nb - 1];"),
    ("matched gradient drops the filter partial", "for (int e = 0; e < 2 * n; ++e) g_ri[e] += gh[e];",
     "for (int e = 0; e < 2 * n; ++e) g_ri[e] += 0.0 * gh[e];"),
    ("threshold gradient sign", "grho[i] += gy * (-a * c * (1.0 - t * t));", "grho[i] += gy * (a * c * (1.0 - t * t));"),
    ("Eq. 42 weights swapped", "terms[0] = c->eps * lw + (1.0 - c->eps) * ls;",
     "terms[0] = (1.0 - c->eps) * lw + c->eps * ls;"),
    ("L_SNRL absolute instead of squared", "ls += (pm - ptar) * (pm - ptar);", "ls += fabs(pm - ptar);"),
    ("sampled-cell decode with d and j swapped", "int j = (int)(id % L);\n        int d = (int)((id / L) % D);",
     "int j = (int)((id / D) % L);\n        int d = (int)(id % D);"),
    ("rank-one filter update without the conjugate", "? x[(size_t)m * N + n] * conj(delta) : 0.0;",
     "? x[(size_t)m * N + n] * delta : 0.0;"),
    ("rank-one waveform update at the wrong sample's phasor", "for (int j = 0; j < L; ++j) ej[j] = E[(size_t)j * N + n0];",
     "for (int j = 0; j < L; ++j) ej[j] = E[(size_t)j * N];"),
    ("rank-one update keeps the unperturbed peak of a touched pair",
     "const fd_stat* s = touched ? &pert[((size_t)ci * 2 + side) * P + pair] : &base[pair];",
     "const fd_stat* s = &base[pair];"),
    ("soft-quantizer derivative 1 - t", "ds += a * c * (1.0 - t * t);", "ds += a * c * (1.0 - t);"),
    ("thresholds i/K", "rho[i] = ((double)i + 0.5) / (double)K;", "rho[i] = (double)i / (double)K;"),
    ("Adam second moment of g, not g^2", "v[e] = b2 * v[e] + (1.0 - b2) * g[e] * g[e];",
     "v[e] = b2 * v[e] + (1.0 - b2) * fabs(g[e]);"),
    ("projection without clipping", "double v = val[b] < 0.0 ? 0.0 : (val[b] > 1.0 ? 1.0 : val[b]);",
     "double v = val[b];"),
    ("PSLR normalised by sqrt(N)", "out[0] = 20.0 * log10(psl[0] / (double)N);",
     "out[0] = 20.0 * log10(psl[0] / sqrt((double)N));"),
    ("acceptance PSL ignores the weight map", "if (w && !(w[(size_t)d * L + j] > 0)) continue;", ""),
    ("p-norm without the 1/p root", "if (c->pnorm > 0) return p->vmax * pow(p->psum, 1.0 / c->pnorm);",
     "if (c->pnorm > 0) return p->vmax * p->psum;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {name}"
    mutated = tmp_path / "sqngd_oracle.c"
    mutated.write_text(src.replace(old, new))
    env = dict(os.environ, SQNGD_ORACLE_SOURCE=str(mutated), SQNGD_ORACLE_BUILD=str(tmp_path / "build"),
               PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught: {name}\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout or "error" in r.stdout.lower()


RN_SRC = os.path.join(ROOT, "oracle", "resnet_oracle.py")
RN_MUTATIONS = [
    ("tanh derivative 1 - h", "ds = dh * (1.0 - h * h)", "ds = dh * (1.0 - h)"),
    ("skip path dropped in the backward pass", "dh = ds + W1.T @ dq", "dh = W1.T @ dq"),
    ("skip path dropped in the forward pass", "h = np.tanh(h + W2 @ r + b2)", "h = np.tanh(W2 @ r + b2)"),
    ("first-layer gradient transposed", "g[2 + 4 * k] = np.outer(dq, h_prev)", "g[2 + 4 * k] = np.outer(h_prev, dq)"),
    ("Adam without bias correction", "theta -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)",
     "theta -= lr * m / (np.sqrt(v) + eps)"),
    ("output bias not the logit of z0", "parts.append(np.log(z / (1.0 - z)))", "parts.append(np.log(z))"),
]


@pytest.mark.parametrize("name,old,new", RN_MUTATIONS, ids=[m[0] for m in RN_MUTATIONS])
def test_generator_pins_catch_planted_mistake(tmp_path, name, old, new):
    """The same for the ResNet generator's oracle: its pins, run against a
    mutated copy, must fail."""
    import importlib.util

    import tests.test_resnet_oracle as pins
    src = open(RN_SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {name}"
    path = tmp_path / "resnet_oracle_mut.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("resnet_oracle_mut", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    saved = pins.rn
    pins.rn = mod
    caught = []
    try:
        for fn in (pins.test_gradient_matches_finite_differences, pins.test_initial_output_is_z0,
                   pins.test_zero_blocks_are_identity_through_tanh, pins.test_adam_matches_torch):
            try:
                fn()
            except (AssertionError, pytest.skip.Exception) as e:
                if isinstance(e, AssertionError):
                    caught.append(fn.__name__)
    finally:
        pins.rn = saved
    assert caught, f"no pin caught: {name}"


WS_SRC = os.path.join(ROOT, "oracle", "warmstart_oracle.py")
WS_MUTATIONS = [
    ("convolution tap reversed", "z += W[:, :, t] @ hp[:, t:t + N]", "z += W[:, :, kw - 1 - t] @ hp[:, t:t + N]"),
    ("softmax gradient without the target", "p[t, np.arange(N)] -= 1.0", "p[t, np.arange(N)] -= 0.0"),
    ("input gradient with the forward tap order", "gh += W[:, :, t].T @ gp[:, 2 * pad - t:2 * pad - t + N]",
     "gh += W[:, :, t].T @ gp[:, t:t + N]"),
    ("tanh derivative 1 - h", "g = gh * (1.0 - hs[li] ** 2)", "g = gh * (1.0 - hs[li])"),
    ("loss not averaged over elements", "scale = 1.0 / (M * N)", "scale = 1.0 / M"),
    ("Adam without bias correction", "mh = m_ / (1 - b1 ** t)", "mh = m_"),
]


@pytest.mark.parametrize("name,old,new", WS_MUTATIONS, ids=[m[0] for m in WS_MUTATIONS])
def test_warmstart_pins_catch_planted_mistake(tmp_path, name, old, new):
    """The same for the warm-start network's oracle."""
    import importlib.util

    import tests.test_warmstart_oracle as pins
    src = open(WS_SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {name}"
    path = tmp_path / "warmstart_oracle_mut.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("warmstart_oracle_mut", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    saved = pins.wo
    pins.wo = mod
    caught = []
    try:
        for nm in dir(pins):
            fn = getattr(pins, nm)
            if not (nm.startswith("test_") and callable(fn)):
                continue
            try:
                fn()
            except AssertionError:
                caught.append(nm)
            except pytest.skip.Exception:
                pass
    finally:
        pins.wo = saved
    assert caught, f"no pin caught: {name}"
