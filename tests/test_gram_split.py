"""The operand splitting of the tensor-core Gram blocks (Ozaki-style error-free
transformation, as documented in the kernel): a model of its integer arithmetic on the host
that checks the facts the kernel's exactness rests on.

* F = round(|x| 2^(42 - e)) with |x| < 2^e is at most 2^42, and its six balanced base-128
  digits (digit 0 in [0, 128], the others in [-64, 63], obtained from F + 64 (2^28 + 2^21 +
  2^14 + 2^7 + 1)) reconstruct F exactly;
* every digit and every product of two digits is exact in BF16 / FP32;
* for every group g = s + t <= 6 (0-based) the sum of digit products over 512 reals stays
  within 2^24, so an FP32 accumulator holds it exactly;
* the split dot product (groups up to 6, FP64 above) is within 2^-42 sqrt(K) of
  max|a| max|b| of the exact dot product of random data.
"""
import math
from fractions import Fraction

import numpy as np

BIAS = 64 * ((1 << 28) + (1 << 21) + (1 << 14) + (1 << 7) + 1)


def fixed(x, e):
    """round(|x| 2^(42 - e)) from the IEEE double's fields (ties up)."""
    m, ex = math.frexp(abs(x))          # |x| = m 2^ex, 0.5 <= m < 1
    if m == 0.0:
        return 0
    mant = int(m * (1 << 53))           # 53-bit integer
    sh = 53 - 42 + e - ex               # |x| 2^(42-e) = mant 2^-(sh)
    if sh <= 0:
        return mant << -sh
    if sh > 64:
        return 0
    return ((mant >> (sh - 1)) + 1) >> 1


def digits(F):
    g = F + BIAS
    return [g >> 35] + [((g >> (35 - 7 * s)) & 127) - 64 for s in range(1, 6)]


def exponent_of(v):
    return max(math.frexp(abs(x))[1] for x in v if x != 0.0)


def test_digits_reconstruct_and_stay_in_range():
    rng = np.random.default_rng(5)
    for scale in (1e-30, 1.0, 3e17):
        v = rng.standard_normal(4000) * scale
        e = exponent_of(v)
        for x in v:
            assert abs(x) < 2.0 ** e
            F = fixed(x, e)
            assert F <= 1 << 42
            d = digits(F)
            assert 0 <= d[0] <= 128 and all(-64 <= t <= 63 for t in d[1:])
            assert sum(t * (1 << (35 - 7 * s)) for s, t in enumerate(d)) == F
            # representation error at most half a unit of 2^(e - 42)
            assert abs(Fraction(F, 1 << 42) * Fraction(2) ** e - Fraction(abs(x))) <= Fraction(2) ** (e - 43)
    # the largest digits the splitting produces
    assert digits(1 << 42) == [128, 0, 0, 0, 0, 0]


def test_group_sums_fit_fp32():
    dmax = [128] + [64] * 5
    for g in range(7):
        bound = sum(dmax[s] * dmax[g - s] for s in range(6) if 0 <= g - s < 6) * 512
        assert bound <= 1 << 24, (g, bound)
    # the products and partial sums are exact in FP32
    for a in (-64, 63, 128):
        for b in (-64, 63, 128):
            assert float(np.float32(a * b)) == a * b


def test_split_dot_product_accuracy():
    rng = np.random.default_rng(6)
    K = 4096
    a = rng.standard_normal(K)
    b = rng.standard_normal(K)
    ea, eb = exponent_of(a), exponent_of(b)
    da = np.array([digits(fixed(x, ea)) for x in a], dtype=np.int64) * np.sign(a).astype(np.int64)[:, None]
    db = np.array([digits(fixed(x, eb)) for x in b], dtype=np.int64) * np.sign(b).astype(np.int64)[:, None]
    total = Fraction(0)
    for c0 in range(0, K, 512):                       # exact integer group sums per chunk
        for g in range(7):
            sg = 0
            for s in range(6):
                t = g - s
                if 0 <= t < 6:
                    sg += int(np.dot(da[c0:c0 + 512, s], db[c0:c0 + 512, t]))
            assert abs(sg) <= 1 << 24
            total += Fraction(sg) / Fraction(1 << (7 * (g + 2)))
    got = float(total * Fraction(2) ** (ea + eb))
    exact = sum(Fraction(x) * Fraction(y) for x, y in zip(a, b))
    err = abs(Fraction(got) - exact)
    bound = Fraction(2) ** (-42) * math.sqrt(K) * Fraction(2) ** (ea + eb)
    assert err <= bound
    assert float(err) / (np.linalg.norm(a) * np.linalg.norm(b)) < 2e-14
