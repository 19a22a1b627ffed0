// Host-side numerics of liboverlap (FP64, no GPU):
//  * Jacobi elliptic sn, cn by the arithmetic-geometric mean and descending
//    Landen transformation (Abramowitz & Stegun 16.4), complete integral K(m).
//  * Zolotarev coefficients of eps(x) = sum_i omega_i x/(x^2 + sigma_i) on
//    a < |x| < b (Sec. 3): c_l = sn^2/cn^2 (l K'/(2n); k'), k' = sqrt(1-(a/b)^2),
//    product form d y prod(y^2+c_{2l}) / prod(y^2+c_{2l-1}) in y = x/a, d from
//    equioscillation, partial fractions in x.
//  * Small dense complex linear algebra for the Ritz step and the deflation
//    projections: Cholesky, triangular inverse, Hermitian eigensolver (Householder
//    tridiagonalisation and implicit QR; cyclic Jacobi as its fallback), LU solve;
//    Sturm bisection for tridiagonal extremes (Lanczos).
#include "hostmath.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <limits>
#include <vector>

namespace ovl {

// ------------------------------------------------------------------ elliptic
// The complement mc = 1 - m is passed on its own: for m within rounding of 1 (the Zolotarev
// modulus k' = sqrt(1 - (a/b)^2) at large b/a) 1 - m in double would lose it entirely.
static void agm_phi(double u, double m, double mc, double* phi_out, double* K_out) {
  // A&S 16.4: a0 = 1, b0 = sqrt(1-m), c0 = sqrt(m)
  double a[64], c[64];
  a[0] = 1.0;
  double b = std::sqrt(mc);
  c[0] = std::sqrt(m);
  int N = 0;
  while (N < 60) {
    const double an = 0.5 * (a[N] + b);
    const double cn = 0.5 * (a[N] - b);
    b = std::sqrt(a[N] * b);
    ++N;
    a[N] = an;
    c[N] = cn;
    if (std::fabs(cn) <= 1e-17 * an) break;
  }
  double phi = std::ldexp(a[N] * u, N);
  for (int n = N; n >= 1; --n) phi = 0.5 * (phi + std::asin(c[n] / a[n] * std::sin(phi)));
  if (phi_out) *phi_out = phi;
  if (K_out) *K_out = M_PI / (2.0 * a[N]);
}

double ellip_K(double m, double mc) {
  double K;
  agm_phi(0.0, m, mc, nullptr, &K);
  return K;
}

void ellip_sncn(double u, double m, double mc, double* sn, double* cn) {
  double phi;
  agm_phi(u, m, mc, &phi, nullptr);
  *sn = std::sin(phi);
  *cn = std::cos(phi);
}

// ------------------------------------------------------------------ Zolotarev
// R0(y) = y prod_{l<n} (y^2 + c_{2l}) / prod_{l<=n} (y^2 + c_{2l-1}), evaluated as
// y / (y^2 + c_{2n-1}) times the n-1 ratios (y^2 + c_{2l}) / (y^2 + c_{2l-1}): the two
// products on their own leave the double range (n factors up to (b/a)^2 each, e.g.
// n = 64 at b/a = 2600), the ratios stay between 1 and c_{2l} / c_{2l-1}.
static double r0(double y, const std::vector<double>& c, int n) {
  const double y2 = y * y;
  double r = y / (y2 + c[2 * n - 2]);
  for (int l = 1; l < n; ++l) r *= (y2 + c[2 * l - 1]) / (y2 + c[2 * l - 2]);
  return r;
}

int zolotarev_coeffs(int n, double a, double b, double* omega, double* sigma, double* delta) {
  if (n < 1 || !(a > 0) || !(b > a)) return -1;
  const double k = a / b;          // the complementary modulus of k'
  const double mc = k * k;         // 1 - k'^2, exact up to one rounding
  if (!(mc > 0)) return -1;
  const double m1 = 1.0 - mc;
  const double Kp = ellip_K(m1, mc);
  std::vector<double> c(2 * n - 1);
  for (int l = 1; l <= 2 * n - 1; ++l) {
    double sn, cn;
    if (l <= n) {
      ellip_sncn(l * Kp / (2.0 * n), m1, mc, &sn, &cn);
      c[l - 1] = (sn * sn) / (cn * cn);
    } else {
      // past K'/2 cn(u) is small and cos(am u) loses it: with delta = K' - u,
      // sn(K' - delta) / cn(K' - delta) = cn(delta) / (k sn(delta)) (the quarter-period shift
      // sn(u + K') = cd(u), cn(u + K') = -k sd(u))
      ellip_sncn((2 * n - l) * Kp / (2.0 * n), m1, mc, &sn, &cn);
      const double t = cn / (k * sn);
      c[l - 1] = t * t;
    }
  }
  // extrema of R0 over y in [1, b/a]: endpoints plus golden-section refinement of
  // every interior extremum of a dense logarithmic grid
  const double ly = std::log(b / a);
  const int G = 8000 + 400 * n;
  std::vector<double> v(G + 1);
  for (int k = 0; k <= G; ++k) v[k] = r0(std::exp(ly * k / G), c, n);
  double lo = std::min(v[0], v[G]), hi = std::max(v[0], v[G]);
  const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
  for (int k = 1; k < G; ++k) {
    const bool isMax = v[k] >= v[k - 1] && v[k] >= v[k + 1];
    const bool isMin = v[k] <= v[k - 1] && v[k] <= v[k + 1];
    if (!isMax && !isMin) continue;
    const double sgn = isMax ? 1.0 : -1.0;
    double l = ly * (k - 1) / G, r = ly * (k + 1) / G;
    for (int it = 0; it < 200 && r - l > 1e-15 * (1.0 + std::fabs(r)); ++it) {
      const double x1 = r - gr * (r - l), x2 = l + gr * (r - l);
      if (sgn * r0(std::exp(x1), c, n) > sgn * r0(std::exp(x2), c, n)) r = x2;
      else l = x1;
    }
    const double e = r0(std::exp(0.5 * (l + r)), c, n);
    if (isMax) hi = std::max(hi, std::max(e, v[k]));
    else lo = std::min(lo, std::min(e, v[k]));
  }
  const double d = 2.0 / (lo + hi);
  *delta = (hi - lo) / (hi + lo);
  // omega_i = a d prod_{l<n} (c_{2l} - c_{2i-1}) / prod_{l!=i} (c_{2l-1} - c_{2i-1}) with the
  // n-1 factors of numerator and denominator paired in index order: c is increasing, so
  // every ratio lies in (0, 1) and neither product can overflow (they do for n near 50)
  for (int i = 0; i < n; ++i) {
    const double ci = c[2 * i];
    double ratio = 1.0;
    for (int l = 1; l < n; ++l) {
      const int j = (l - 1 < i) ? l - 1 : l;   // the l-th index of {0 .. n-1} without i
      ratio *= (c[2 * l - 1] - ci) / (c[2 * j] - ci);
    }
    omega[i] = a * d * ratio;
    sigma[i] = a * a * ci;
    if (!std::isfinite(omega[i]) || !std::isfinite(sigma[i])) return -1;
  }
  return std::isfinite(*delta) ? 0 : -1;
}

double pole_gbound(double sigma, double a, double b) {
  const double r = std::sqrt(sigma);
  if (r >= a && r <= b) return 0.5 / r;
  if (r < a) return a / (a * a + sigma);
  return b / (b * b + sigma);
}

// ------------------------------------------------------------------ dense
using cd = std::complex<double>;

int cholesky_lower(int n, cd* A /* row-major, in: Hermitian PD, out: L */) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(A[j * n + k]);
    if (!(d > 0.0)) return -1;
    const double ljj = std::sqrt(d);
    A[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      cd s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * std::conj(A[j * n + k]);
      A[i * n + j] = s / ljj;
    }
    for (int k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
  }
  return 0;
}

void lower_inverse(int n, const cd* L, cd* Li) {
  for (int i = 0; i < n * n; ++i) Li[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    Li[j * n + j] = 1.0 / L[j * n + j];
    for (int i = j + 1; i < n; ++i) {
      cd s = 0.0;
      for (int k = j; k < i; ++k) s += L[i * n + k] * Li[k * n + j];
      Li[i * n + j] = -s / L[i * n + i];
    }
  }
}

void eigh_jacobi(int n, cd* A /* Hermitian, destroyed */, double* w, cd* Z /* columns */) {
  for (int i = 0; i < n * n; ++i) Z[i] = 0.0;
  for (int i = 0; i < n; ++i) Z[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int p = 0; p < n; ++p) {
      diag += std::norm(A[p * n + p]);
      for (int q = p + 1; q < n; ++q) off += std::norm(A[p * n + q]);
    }
    if (off <= 1e-32 * (diag + 1e-300)) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const cd apq = A[p * n + q];
        const double c_abs = std::abs(apq);
        if (c_abs < 1e-300) continue;
        // phase: make A[p][q] real positive by scaling column/row q by conj(u)
        const cd u = apq / c_abs;
        for (int r = 0; r < n; ++r) {
          A[r * n + q] *= std::conj(u);
        }
        for (int r = 0; r < n; ++r) {
          A[q * n + r] *= u;
        }
        for (int r = 0; r < n; ++r) Z[r * n + q] *= std::conj(u);
        const double app = A[p * n + p].real(), aqq = A[q * n + q].real();
        const double theta = (aqq - app) / (2.0 * c_abs);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int r = 0; r < n; ++r) {
          const cd arp = A[r * n + p], arq = A[r * n + q];
          A[r * n + p] = cs * arp - sn * arq;
          A[r * n + q] = sn * arp + cs * arq;
        }
        for (int r = 0; r < n; ++r) {
          const cd apr = A[p * n + r], aqr = A[q * n + r];
          A[p * n + r] = cs * apr - sn * aqr;
          A[q * n + r] = sn * apr + cs * aqr;
        }
        A[p * n + q] = 0.0;
        A[q * n + p] = 0.0;
        A[p * n + p] = A[p * n + p].real();
        A[q * n + q] = A[q * n + q].real();
        for (int r = 0; r < n; ++r) {
          const cd zrp = Z[r * n + p], zrq = Z[r * n + q];
          Z[r * n + p] = cs * zrp - sn * zrq;
          Z[r * n + q] = sn * zrp + cs * zrq;
        }
      }
    }
  }
  // sort ascending
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int x, int y) { return A[x * n + x].real() < A[y * n + y].real(); });
  std::vector<cd> Zs(n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[idx[j] * n + idx[j]].real();
    for (int r = 0; r < n; ++r) Zs[r * n + j] = Z[r * n + idx[j]];
  }
  for (int i = 0; i < n * n; ++i) Z[i] = Zs[i];
}

// Real symmetric tridiagonal eigenproblem by implicit symmetric QR steps with Wilkinson
// shifts (Golub & Van Loan, Matrix Computations, 8.3): on the last unreduced block
// [p, q] a rotation of rows/columns (p, p+1) made from (a_p - mu, b_p) starts a bulge
// that further rotations chase to the bottom; off-diagonals below eps (|a_i| + |a_i+1|)
// are set to zero. a: diagonal, b: b[i] couples i and i+1. Every rotation is applied to
// the columns of Z (n x n row-major). false if some block has not converged after
// 30 n steps in all.
static bool tridiag_qr(int n, double* a, double* b, cd* Z) {
  const double eps = std::numeric_limits<double>::epsilon();
  int q = n - 1, steps = 0;
  while (q > 0) {
    if (std::fabs(b[q - 1]) <= eps * (std::fabs(a[q - 1]) + std::fabs(a[q]))) {
      b[q - 1] = 0.0;
      --q;
      continue;
    }
    int p = q - 1;
    while (p > 0 && std::fabs(b[p - 1]) > eps * (std::fabs(a[p - 1]) + std::fabs(a[p]))) --p;
    if (p > 0) b[p - 1] = 0.0;
    if (++steps > 30 * n) return false;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer to a_q
    const double d = 0.5 * (a[q - 1] - a[q]), bq = b[q - 1];
    const double mu = a[q] - bq * bq / (d + std::copysign(std::hypot(d, bq), d));
    double x = a[p] - mu, z = b[p];
    for (int k = p; k < q; ++k) {
      // P = [[c, -s], [s, c]] on coordinates (k, k+1), P^T (x, z) = (r, 0)
      const double r = std::hypot(x, z);
      const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? z / r : 0.0;
      if (k > p) b[k - 1] = r;                                  // the bulge is gone
      const double ak = a[k], ak1 = a[k + 1], bk = b[k];
      a[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
      a[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
      b[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
      double bulge = 0.0;
      if (k + 1 < q) {
        bulge = s * b[k + 1];                                   // new entry (k, k+2)
        b[k + 1] = c * b[k + 1];
      }
      for (int i = 0; i < n; ++i) {
        const cd zk = Z[(size_t)i * n + k], zk1 = Z[(size_t)i * n + k + 1];
        Z[(size_t)i * n + k] = c * zk + s * zk1;
        Z[(size_t)i * n + k + 1] = -s * zk + c * zk1;
      }
      x = b[k];
      z = bulge;
    }
  }
  return true;
}

// Hermitian eigendecomposition: Householder reduction to tridiagonal form (Golub & Van
// Loan 8.3.1; reflections I - tau v v^dag chosen so that no cancellation occurs in v_0,
// each applied as the rank-2 update A - v w^dag - w v^dag and accumulated in Q), a diagonal
// phase D that makes the off-diagonal real and non-negative (T = D T' D^dag), then
// tridiag_qr on T' with the columns of Q D. Cyclic Jacobi is the fallback should the QR
// iteration not converge. w ascending, Z the eigenvectors as columns.
void eigh_herm(int n, cd* A /* Hermitian, destroyed */, double* w, cd* Z /* columns */) {
  if (n <= 0) return;
  std::vector<cd> Q((size_t)n * n, 0.0), v(n), pv(n);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  const std::vector<cd> A0(A, A + (size_t)n * n);
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;   // reflect x = A[k+1 .., k]
    double sig = 0.0;
    for (int i = 1; i < L; ++i) sig += std::norm(A[(size_t)(k + 1 + i) * n + k]);
    if (sig == 0.0) continue;
    const cd x0 = A[(size_t)(k + 1) * n + k];
    const double ax0 = std::abs(x0), nx = std::sqrt(ax0 * ax0 + sig);
    const cd ph = ax0 > 0.0 ? x0 / ax0 : cd(1.0);
    const cd beta = -ph * nx;                       // H x = beta e_1
    for (int i = 0; i < L; ++i) v[i] = A[(size_t)(k + 1 + i) * n + k];
    v[0] = x0 - beta;                               // = ph (|x0| + ||x||)
    double vv = 0.0;
    for (int i = 0; i < L; ++i) vv += std::norm(v[i]);
    const double tau = 2.0 / vv;
    // p = tau A22 v, K = tau/2 v^dag p (real), w = p - K v, A22 -= v w^dag + w v^dag
    for (int i = 0; i < L; ++i) {
      cd t = 0.0;
      const cd* row = A + (size_t)(k + 1 + i) * n + (k + 1);
      for (int j = 0; j < L; ++j) t += row[j] * v[j];
      pv[i] = tau * t;
    }
    cd K = 0.0;
    for (int i = 0; i < L; ++i) K += std::conj(v[i]) * pv[i];
    K *= 0.5 * tau;
    for (int i = 0; i < L; ++i) pv[i] -= K.real() * v[i];
    for (int i = 0; i < L; ++i) {
      cd* row = A + (size_t)(k + 1 + i) * n + (k + 1);
      for (int j = 0; j < L; ++j) row[j] -= v[i] * std::conj(pv[j]) + pv[i] * std::conj(v[j]);
    }
    A[(size_t)(k + 1) * n + k] = beta;
    A[(size_t)k * n + k + 1] = std::conj(beta);
    for (int i = 1; i < L; ++i) {
      A[(size_t)(k + 1 + i) * n + k] = 0.0;
      A[(size_t)k * n + k + 1 + i] = 0.0;
    }
    // Q <- Q H = Q - tau (Q v) v^dag on columns k+1 ..
    for (int r = 0; r < n; ++r) {
      cd* row = Q.data() + (size_t)r * n + (k + 1);
      cd t = 0.0;
      for (int j = 0; j < L; ++j) t += row[j] * v[j];
      t *= tau;
      for (int j = 0; j < L; ++j) row[j] -= t * std::conj(v[j]);
    }
  }
  std::vector<double> a(n), b(std::max(1, n - 1), 0.0);
  std::vector<cd> ph(n, 1.0);
  for (int i = 0; i < n; ++i) a[i] = A[(size_t)i * n + i].real();
  for (int i = 0; i + 1 < n; ++i) {
    const cd e = A[(size_t)(i + 1) * n + i];
    const double ae = std::abs(e);
    b[i] = ae;
    ph[i + 1] = ae > 0.0 ? ph[i] * (e / ae) : ph[i];
  }
  for (int r = 0; r < n; ++r)
    for (int j = 0; j < n; ++j) Z[(size_t)r * n + j] = Q[(size_t)r * n + j] * ph[j];
  if (!tridiag_qr(n, a.data(), b.data(), Z)) {
    std::vector<cd> Ac = A0;
    eigh_jacobi(n, Ac.data(), w, Z);
    return;
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return a[x] < a[y]; });
  std::vector<cd> Zs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = a[idx[j]];
    for (int r = 0; r < n; ++r) Zs[(size_t)r * n + j] = Z[(size_t)r * n + idx[j]];
  }
  std::copy(Zs.begin(), Zs.end(), Z);
}

int lu_solve(int n, cd* A, cd* B, int nb) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::abs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A[i * n + k]) > best) {
        best = std::abs(A[i * n + k]);
        p = i;
      }
    if (best == 0.0) return -1;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      for (int j = 0; j < nb; ++j) std::swap(B[k * nb + j], B[p * nb + j]);
    }
    for (int i = k + 1; i < n; ++i) {
      const cd f = A[i * n + k] / A[k * n + k];
      A[i * n + k] = f;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      for (int j = 0; j < nb; ++j) B[i * nb + j] -= f * B[k * nb + j];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int j = 0; j < nb; ++j) {
      cd s = B[k * nb + j];
      for (int i = k + 1; i < n; ++i) s -= A[k * n + i] * B[i * nb + j];
      B[k * nb + j] = s / A[k * n + k];
    }
  }
  return 0;
}

// number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm count)
static int sturm(int n, const double* d, const double* e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < n; ++i) {
    const double e2 = i > 0 ? e[i - 1] * e[i - 1] : 0.0;
    q = d[i] - x - (i > 0 ? e2 / q : 0.0);
    if (q == 0.0) q = 1e-300;
    if (q < 0) ++cnt;
  }
  return cnt;
}

void tridiag_extremes(int n, const double* d, const double* e, double* lmin, double* lmax) {
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  double a = lo, b = hi;
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (a + b);
    if (sturm(n, d, e, m) >= 1) b = m;
    else a = m;
  }
  *lmin = 0.5 * (a + b);
  a = lo;
  b = hi;
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (a + b);
    if (sturm(n, d, e, m) >= n) b = m;
    else a = m;
  }
  *lmax = 0.5 * (a + b);
}

}  // namespace ovl
