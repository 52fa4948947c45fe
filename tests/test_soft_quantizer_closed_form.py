"""The closed form that the GPU path uses for Eq. 24 with uniform thresholds,
restated here in FP64 and checked against the oracle's sum of all K tanh terms.

For rho_i = (i + 1/2)/K and a_i = a, tanh(u) + 1 = 2 s(2u) (s the logistic
function) turns the sum into y = 2a S(z), S = sum_{i<K} s(alpha (x - i)) with
alpha = 2c/K and x = zK - 1/2: a smooth function summed at unit spacing.  The
midpoint Euler-Maclaurin formula over [-1/2, K - 1/2] gives

    S = zK + [sp(-v0) - sp(v1)]/alpha + (alpha/24)[d1(v1) - d1(v0)]
          - (7 alpha^3/5760)[d3(v1) - d3(v0)],

v0 = 2cz, v1 = 2c(z - 1), sp the softplus, d1 = s(1 - s), d3 = d1(1 - 6 d1),
and dS/dz from the same terms differentiated.  The remainder is of order
e^{-2 pi^2/alpha} plus the next end term, so for alpha <= 1/2 the formula must
match the direct sum far below FP32 resolution (here: 1e-7 on y, 1e-6
relative on Q_A'), at the ends of [0, 1] as well as inside.  A wrong sign or a
missing end term fails by orders of magnitude more.  CPU only: the oracle is
the reference, the GPU kernels are not involved.
"""
import numpy as np
import pytest

from paper_2604_25728_gb300 import workloads as wl


def _closed(z, K, a, c):
    al = 2.0 * c / K
    v0, v1 = 2.0 * c * z, 2.0 * c * (z - 1.0)

    def sp(w):
        return np.maximum(w, 0.0) + np.log1p(np.exp(-np.abs(w)))

    def sig(v):
        e = np.exp(-np.abs(v))
        return np.where(v >= 0, 1.0 / (1.0 + e), e / (1.0 + e))

    s0, s1 = sig(v0), sig(v1)
    d0, d1 = s0 * (1 - s0), s1 * (1 - s1)
    k1, k3 = al / 24.0, 7.0 * al ** 3 / 5760.0
    S = z * K + (sp(-v0) - sp(v1)) / al + k1 * (d1 - d0) - k3 * (d1 * (1 - 6 * d1) - d0 * (1 - 6 * d0))
    g0, g1 = d0 * (1 - 2 * s0), d1 * (1 - 2 * s1)
    dS = K * (s0 - s1) + 2.0 * c * (k1 * (g1 - g0) - k3 * (g1 * (1 - 12 * d1) - g0 * (1 - 12 * d0)))
    return 2.0 * a * S, 2.0 * a * dS


@pytest.mark.parametrize("B,r_n,c", [(16, 100, 300.0), (64, 100, 300.0), (8, 100, 100.0), (8, 200, 300.0)])
def test_closed_form_matches_the_oracle_sum(orc, B, r_n, c):
    rho, a = orc.thresholds(B, r_n)
    K = B * r_n
    assert 2.0 * c / K <= 0.5                       # the range where the GPU path uses it
    u = wl.uniform(31, 1500, 2)
    z = np.concatenate([u[:1000], 0.03 * u[1000:1250], 1.0 - 0.03 * u[1250:], [0.0, 1.0, 1e-6, 1.0 - 1e-6]])
    y, dy = orc.soft_quantize(z, rho, a, c)
    yc, dyc = _closed(z, K, a, c)
    assert np.max(np.abs(yc - y)) <= 1e-7
    assert np.max(np.abs(dyc - dy)) <= 1e-6 * np.max(np.abs(dy))


def test_a_missing_end_term_is_detected(orc):
    """Without the first Euler-Maclaurin end term the formula is off near the
    ends of [0, 1] by far more than the bar above: the test has teeth."""
    B, r_n, c = 16, 100, 300.0
    rho, a = orc.thresholds(B, r_n)
    K = B * r_n
    z = np.linspace(0.0, 0.02, 200)
    y, _ = orc.soft_quantize(z, rho, a, c)
    al = 2.0 * c / K
    yc, _ = _closed(z, K, a, c)
    s0 = 1.0 / (1.0 + np.exp(-2.0 * c * z))
    d0 = s0 * (1 - s0)
    y_wrong = yc + 2.0 * a * (al / 24.0) * d0        # drop the k1 term at the lower end
    assert np.max(np.abs(yc - y)) <= 1e-7
    assert np.max(np.abs(y_wrong - y)) > 1e-5
