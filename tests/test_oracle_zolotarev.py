"""Pins of the oracle's Zolotarev table: Chebyshev alternation (2n+1 extrema of 1 - R with
equal magnitude and alternating sign characterise the minmax rational approximation of
sign(x) on [sqrt(eps), 1]), oddness, the uniform bound |R - sign| <= delta (Sec. 2.2's
uniform error statement, carried over to the rational form) and monotonicity in n."""
import mpmath as mp
import numpy as np
import pytest

from oracle import zolotarev


@pytest.mark.parametrize("n,eps", [(4, 1e-2), (8, 1e-3), (12, 1e-4), (16, 1e-4)])
def test_alternation(n, eps):
    c = zolotarev.zolotarev(n, eps)
    err = c["extrema_err"]
    assert len(err) == 2 * n + 1
    d = c["delta"]
    for k, e in enumerate(err):
        assert abs(abs(e) - d) <= 1e-8 * d
        if k:
            assert (e > 0) != (err[k - 1] > 0)
    # extrema span the whole interval: endpoints included
    assert abs(c["extrema_x"][0] - np.sqrt(eps)) < 1e-15 and abs(c["extrema_x"][-1] - 1) < 1e-15


@pytest.mark.parametrize("n,eps", [(6, 1e-3), (16, 1e-4)])
def test_uniform_bound_and_oddness(n, eps):
    c = zolotarev.zolotarev(n, eps)
    d = c["delta"]
    xs = np.geomspace(np.sqrt(eps), 1.0, 700)
    worst = 0.0
    for x in xs:
        r = zolotarev.evaluate(c, x)
        worst = max(worst, float(abs(1 - r)))
        assert abs(zolotarev.evaluate(c, -x) + r) < 1e-30
    assert worst <= d * (1 + 1e-9)
    assert worst >= 0.5 * d  # the bound is attained up to grid resolution


def test_shifts_positive_and_delta_decreasing():
    prev = 1.0
    for n in (4, 8, 12, 16, 20):
        c = zolotarev.zolotarev(n, 1e-4)
        assert all(s > 0 for s in c["sigma"]) and all(b > 0 for b in c["b"])
        assert np.all(np.diff(c["sigma"]) > 0)
        assert c["delta"] < prev
        prev = c["delta"]


@pytest.mark.parametrize("eps", [0.5, 0.1, 1e-2, 1e-4])
def test_one_pole_closed_form(eps):
    """n = 1: R(x) = b x / (x^2 + sigma) on [k, 1], k = sqrt(eps).  Equioscillation at x = k, the
    maximum x = sqrt(sigma) and x = 1 gives R(k) = R(1), hence sigma = k, and
    1 - R(1) = R(sqrt(k)) - 1 fixes b = 2 / (1/(1 + k) + 1/(2 k^(1/2))), delta = 1 - b/(1 + k)."""
    z = zolotarev.zolotarev(1, eps)
    k = np.sqrt(eps)
    b = 2.0 / (1.0 / (1.0 + k) + 1.0 / (2.0 * eps ** 0.25))
    assert float(z["sigma"][0]) == pytest.approx(k, rel=1e-14)
    assert float(z["b"][0]) == pytest.approx(b, rel=1e-14)
    assert float(z["delta"]) == pytest.approx(1.0 - b / (1.0 + k), rel=1e-12)
