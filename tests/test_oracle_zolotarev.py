"""Pins of the oracle's Zolotarev coefficients (Sec. 3): the n = 1 closed form,
equioscillation between 1 - Delta and 1 + Delta at 2n+1 alternating points,
monotone Delta, and an independent arbitrary-precision check of the elliptic
functions."""
import numpy as np
import pytest

from oracle import zolotarev as zo


@pytest.mark.parametrize("a,b", [(0.2, 2.5), (0.05, 2.5), (1.0, 7.0)])
def test_n1_closed_form(a, b):
    om, sg, delta = zo.zolotarev(1, a, b)
    A = (a + b) / (2 * np.sqrt(a * b))
    assert np.isclose(sg[0], a * b, rtol=1e-13)
    assert np.isclose(om[0], 2 * (a + b) / (1 + A), rtol=1e-12)
    assert np.isclose(delta, ((np.sqrt(b) - np.sqrt(a)) / (np.sqrt(b) + np.sqrt(a))) ** 2, rtol=1e-12)


@pytest.mark.parametrize("n,a,b", [(2, 0.2, 2.5), (3, 0.2, 2.5), (5, 0.1, 2.5), (6, 0.02, 2.5)])
def test_equioscillation(n, a, b):
    om, sg, delta = zo.zolotarev(n, a, b)
    xs = np.exp(np.linspace(np.log(a), np.log(b), 400001))
    err = zo.epsilon(xs, om, sg) - 1.0
    assert np.max(np.abs(err)) <= delta * (1 + 1e-6)
    # count alternating extrema that reach +-Delta
    ext = [err[0]]
    for k in range(1, len(err) - 1):
        if (err[k] - err[k - 1]) * (err[k + 1] - err[k]) <= 0:
            ext.append(err[k])
    ext.append(err[-1])
    big = [e for e in ext if abs(abs(e) - delta) <= 1e-4 * delta]
    signs = np.sign(big)
    alternations = 1 + int(np.sum(signs[1:] != signs[:-1]))
    assert alternations == 2 * n + 1


def test_delta_monotone_and_odd():
    a, b = 0.2136, 2.483
    ds = [zo.zolotarev(n, a, b)[2] for n in range(1, 12)]
    assert all(d2 < d1 for d1, d2 in zip(ds, ds[1:]))
    om, sg, _ = zo.zolotarev(8, a, b)
    x = np.linspace(0.1, 3, 50)
    assert np.allclose(zo.epsilon(-x, om, sg), -zo.epsilon(x, om, sg))
    assert np.all(sg > 0) and np.all(om > 0)


def test_delta_against_mpmath():
    """Delta recomputed independently in 40-digit arithmetic (mpmath elliptic
    functions and a golden-section search for the interior maxima)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    n, a, b = 4, mp.mpf("0.2"), mp.mpf("2.5")
    m1 = 1 - (a / b) ** 2
    Kp = mp.ellipk(m1)
    c = [mp.ellipfun("sn", l * Kp / (2 * n), m=m1) ** 2 / mp.ellipfun("cn", l * Kp / (2 * n), m=m1) ** 2
         for l in range(1, 2 * n)]

    def R0(y):
        num = mp.mpf(1)
        den = mp.mpf(1)
        for l in range(1, n):
            num *= y * y + c[2 * l - 1]
        for l in range(1, n + 1):
            den *= y * y + c[2 * l - 2]
        return y * num / den

    ymax = b / a
    grid = [mp.e ** (mp.log(ymax) * k / 400) for k in range(401)]
    vals = [R0(y) for y in grid]
    lo = min(vals[0], vals[-1])
    hi = lo
    for k in range(1, 400):
        if vals[k] >= vals[k - 1] and vals[k] >= vals[k + 1]:
            l, r = mp.log(grid[k - 1]), mp.log(grid[k + 1])
            g = (mp.sqrt(5) - 1) / 2
            for _ in range(120):
                m1_, m2_ = r - g * (r - l), l + g * (r - l)
                if R0(mp.e ** m1_) > R0(mp.e ** m2_):
                    r = m2_
                else:
                    l = m1_
            hi = max(hi, R0(mp.e ** ((l + r) / 2)))
    delta_mp = (hi - lo) / (hi + lo)
    got = zo.zolotarev(n, 0.2, 2.5)[2]
    assert abs(got - float(delta_mp)) <= 1e-9 * float(delta_mp)


@pytest.mark.parametrize("n,a,b,rtol", [(7, 0.13, 2.4, 1e-12), (48, 0.002, 2.6, 1e-12), (64, 0.001, 2.6, 1e-12)])
def test_elliptic_values_against_mpmath(n, a, b, rtol):
    """c_l = sn^2/cn^2 (l K'/2n; k') against 40-digit mpmath, also at b/a = 1300 and 2600,
    where 1 - (a/b)^2 formed in double and cn near K' would each cost digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    c = zo.c_coefficients(n, a, b)
    m1 = 1 - mp.mpf(a) ** 2 / mp.mpf(b) ** 2
    Kp = mp.ellipk(m1)
    for l in range(1, 2 * n):
        sn = mp.ellipfun("sn", l * Kp / (2 * n), m=m1)
        cn = mp.ellipfun("cn", l * Kp / (2 * n), m=m1)
        assert abs(float(sn ** 2 / cn ** 2) - c[l - 1]) <= rtol * c[l - 1]


@pytest.mark.parametrize("n,a,b", [(48, 0.002, 2.6), (64, 0.001, 2.6), (64, 0.3, 2.6)])
def test_large_order_stays_finite_and_attains_delta(n, a, b):
    """Up to the library's 64 poles and b/a = 2600: every omega_i and sigma_i finite and
    positive, sigma ascending, and the sampled max |1 - epsilon| on [a, b] equals Delta (the
    bound holds and is attained) to the rounding of the partial-fraction sum in double."""
    om, sg, delta = zo.zolotarev(n, a, b)
    assert np.all(np.isfinite(om)) and np.all(np.isfinite(sg)) and np.isfinite(delta)
    assert np.all(om > 0) and np.all(sg > 0) and np.all(np.diff(sg) > 0)
    xs = np.exp(np.linspace(np.log(a), np.log(b), 400001))
    err = np.max(np.abs(zo.epsilon(xs, om, sg) - 1.0))
    assert abs(err - delta) <= 1e-3 * delta + 2e-14, (err, delta)
