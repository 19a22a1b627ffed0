"""Zolotarev optimal rational approximation to sign(x) on a < |x| < b (Sec. 3):

  epsilon(x) = sum_{i=1}^{N_Z} omega_i x / (x^2 + sigma_i),

with |epsilon| oscillating between 1-Delta and 1+Delta on [a, b]. The paper
does not print the coefficients; it refers to Jacobi elliptic functions. Written
out here in the product form: for y = x/a in [1, b/a], k = a/b, k' = sqrt(1 - k^2),
K' = K(k'),

  c_l = sn^2(l K'/(2n); k') / cn^2(l K'/(2n); k'),   l = 1 .. 2n-1
  R(y) = d * y * prod_{l=1}^{n-1} (y^2 + c_{2l}) / prod_{l=1}^{n} (y^2 + c_{2l-1}),

with d fixed by equioscillation, d = 2 / (min R0 + max R0) over [1, b/a], and
Delta = (max R0 - min R0) / (max R0 + min R0). Partial fractions in x = a*y give
sigma_i = a^2 c_{2i-1} and omega_i = a * d * prod_l (c_{2l} - c_{2i-1})
/ prod_{l != i} (c_{2l-1} - c_{2i-1}).

The extrema of R0 are found numerically (dense logarithmic grid, then bounded
scalar minimisation around every grid extremum). Test infrastructure only.
"""
import numpy as np
from scipy import special, optimize


def c_coefficients(n, a, b):
    """c_1 .. c_{2n-1} (index 0 holds c_1).

    K' = K(k') from the complementary parameter k^2 = (a/b)^2 (scipy's ellipkm1), since
    1 - (a/b)^2 formed in double loses it at large b/a; past K'/2, where cn is small,
    sn/cn at u = K' - delta is cn(delta) / (k sn(delta)) with delta = (2n - l) K'/(2n)
    (the quarter-period shift sn(u + K') = cd(u), cn(u + K') = -k sd(u))."""
    k = a / b
    m1 = 1.0 - k * k                      # parameter m = k'^2 for scipy
    Kp = special.ellipkm1(k * k)          # K(1 - k^2) = K(k')
    l = np.arange(1, 2 * n)
    c = np.empty(2 * n - 1)
    near = l <= n
    sn, cn, dn, ph = special.ellipj(l[near] * Kp / (2 * n), m1)
    c[near] = sn ** 2 / cn ** 2
    sn, cn, dn, ph = special.ellipj((2 * n - l[~near]) * Kp / (2 * n), m1)
    c[~near] = (cn / (k * sn)) ** 2
    return c


def r0(y, c, n):
    """R0(y) = y prod (y^2 + c_{2l}) / prod (y^2 + c_{2l-1}) without the scale d, taken as
    y / (y^2 + c_{2n-1}) times the n-1 ratios (y^2 + c_{2l}) / (y^2 + c_{2l-1}): the two
    products alone leave the double range for large n and b/a (n = 64 at b/a = 2600),
    each ratio lies between 1 and c_{2l} / c_{2l-1}."""
    y = np.asarray(y, dtype=np.float64)
    y2 = y * y
    r = y / (y2 + c[2 * n - 2])                        # c_{2n-1}
    for l in range(1, n):
        r = r * (y2 + c[2 * l - 1]) / (y2 + c[2 * l - 2])   # c_{2l} / c_{2l-1}
    return r


def extrema(n, a, b, c=None, ngrid=20001):
    """(min R0, max R0) over y in [1, b/a]."""
    if c is None:
        c = c_coefficients(n, a, b)
    ymax = b / a
    ys = np.exp(np.linspace(0.0, np.log(ymax), ngrid))
    v = r0(ys, c, n)
    lo = min(v[0], v[-1])
    hi = max(v[0], v[-1])
    for k in range(1, ngrid - 1):
        for sgn in (+1.0, -1.0):
            if sgn * v[k] >= sgn * v[k - 1] and sgn * v[k] >= sgn * v[k + 1]:
                res = optimize.minimize_scalar(lambda t: -sgn * r0(np.exp(t), c, n),
                                               bounds=(np.log(ys[k - 1]), np.log(ys[k + 1])),
                                               method="bounded",
                                               options={"xatol": 1e-14})
                val = r0(np.exp(res.x), c, n)
                val = max(val, v[k]) if sgn > 0 else min(val, v[k])
                hi = max(hi, val) if sgn > 0 else hi
                lo = min(lo, val) if sgn < 0 else lo
    return float(lo), float(hi)


def zolotarev(n, a, b):
    """Return (omega[n], sigma[n], Delta) for epsilon(x) = sum omega x / (x^2 + sigma)."""
    c = c_coefficients(n, a, b)
    lo, hi = extrema(n, a, b, c)
    d = 2.0 / (lo + hi)
    delta = (hi - lo) / (hi + lo)
    codd = c[0::2]                         # c_1, c_3, ..., c_{2n-1}
    ceven = c[1::2]                        # c_2, ..., c_{2n-2}
    omega = np.empty(n)
    for i in range(n):
        # prod_l (c_{2l} - c_{2i-1}) / prod_{l != i} (c_{2l-1} - c_{2i-1}), the n-1 factors of
        # each product paired in index order: c is increasing, so every ratio lies in
        # (0, 1) and neither product overflows (both do for n near 50)
        others = np.delete(codd, i)
        ratio = 1.0
        for num_t, den_t in zip(ceven - codd[i], others - codd[i]):
            ratio *= num_t / den_t
        omega[i] = a * d * ratio
    sigma = a * a * codd
    return omega, sigma, delta


def epsilon(x, omega, sigma):
    """epsilon(x) = sum_i omega_i x / (x^2 + sigma_i), Sec. 3."""
    x = np.asarray(x, dtype=np.float64)
    return sum(w * x / (x * x + s) for w, s in zip(omega, sigma))
