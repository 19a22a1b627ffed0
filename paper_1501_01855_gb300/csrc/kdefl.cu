// Kernel low-mode deflation of the sign function (Sec. 1: sign(K) = sum_i psi_i psi_i^dag
// sign(lambda_i) over the eigenpairs of the Hermitian kernel K; in practice the smallest
// eigenvectors of K are deflated and the approximation covers the rest of the spectrum).
//
// ovl_kernel_deflate finds the n_ev eigenpairs of K with the smallest |lambda| by
// Chebyshev-filtered subspace iteration: a block of m = n_ev + max(8, n_ev) vectors is
// filtered with the Chebyshev polynomial of K^2 (degree up to 24) that is bounded by 1 on [c2, b^2]
// and grows fastest below c2 (c2: the largest Rayleigh quotient of K^2 over the block, so
// that the unwanted part of the spectrum is damped), then a Rayleigh-Ritz step with K itself gives
// orthonormal Ritz vectors, signed eigenvalues and residuals ||K x - theta x||. The block
// stays in FP64; every K application is one multi-system Wilson launch over the block and
// the Gram blocks run on the tensor cores. With the eigenpairs stored, the rational is
// rebuilt on [a', b], a' = 0.95 sqrt(lambda_min) of K^2 restricted to the complement
// (300 Lanczos steps with the eigenvectors projected out at every step), with the fewest
// poles that keep Delta <= eps_sign (or the count the caller asks for); every sign
// application then uses sign(K) v = K [R(K^2) P v + sum_i psi_i (psi_i, v) / |lambda_i|]
// (engine.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>

#include "context.h"
#include "hostmath.h"
#include "solver.h"

namespace ovl {

namespace {

// The host part of the Rayleigh-Ritz step of K (Sec. 1 eigenpairs) on the span of m vectors
// X: from E = (x_i, x_j) and H = (x_i, K x_j) (row-major), the coefficients C (m x m) with
// X C orthonormal and C^dag H C = diag(theta), theta in the order of |theta|. OVL_EBREAKDOWN
// when E has no Cholesky factor (the block lost linear independence).
ovl_status kd_rayleigh_ritz_host(int m, std::vector<cd> E, std::vector<cd> H, std::vector<double>& theta,
                                 std::vector<cd>& C) {
  // B = L^-dag with E = L L^dag, so that B^dag E B = 1
  std::vector<cd> L = E;
  if (cholesky_lower(m, L.data()) != 0) return OVL_EBREAKDOWN;
  std::vector<cd> Li((size_t)m * m), B((size_t)m * m);
  lower_inverse(m, L.data(), Li.data());
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) B[(size_t)i * m + j] = std::conj(Li[(size_t)j * m + i]);
  // T = B^dag H B (Hermitian up to rounding: symmetrised)
  std::vector<cd> HB((size_t)m * m), T((size_t)m * m), Z((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      cd s = 0;
      for (int l = 0; l < m; ++l) s += H[(size_t)i * m + l] * B[(size_t)l * m + j];
      HB[(size_t)i * m + j] = s;
    }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      cd s = 0;
      for (int l = 0; l < m; ++l) s += std::conj(B[(size_t)l * m + i]) * HB[(size_t)l * m + j];
      T[(size_t)i * m + j] = s;
    }
  for (int i = 0; i < m; ++i)
    for (int j = i; j < m; ++j) {
      const cd a = 0.5 * (T[(size_t)i * m + j] + std::conj(T[(size_t)j * m + i]));
      T[(size_t)i * m + j] = a;
      T[(size_t)j * m + i] = std::conj(a);
    }
  std::vector<double> w(m);
  eigh_herm(m, T.data(), w.data(), Z.data());
  std::vector<int> ord(m);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return std::fabs(w[x]) < std::fabs(w[y]); });
  // C = B Z, columns in the order of |theta|
  C.assign((size_t)m * m, 0.0);
  theta.resize(m);
  for (int jj = 0; jj < m; ++jj) {
    const int j = ord[jj];
    theta[jj] = w[j];
    for (int i = 0; i < m; ++i) {
      cd s = 0;
      for (int l = 0; l < m; ++l) s += B[(size_t)i * m + l] * Z[(size_t)l * m + j];
      C[(size_t)i * m + jj] = s;
    }
  }
  return OVL_OK;
}

// Rayleigh-Ritz of K on the span of X (m vectors): Xn = X C orthonormal with C^dag (X^dag K X)
// C = diag(theta) (ascending |theta|), KXn = (K X) C, res_i = ||K xn_i - theta_i xn_i||,
// q_i = ||K xn_i||^2 (the Rayleigh quotients of K^2).
ovl_status kd_rayleigh_ritz(ovl_ctx* c, Field& X, Field& KX, Field& Xn, Field& KXn, Field& R, int m,
                            std::vector<double>& theta, std::vector<double>& res, std::vector<double>& q) {
  std::vector<cd> E, H;
  OVL_TRY(gram_host(c, X, 0, m, X, 0, m, 0, E));
  OVL_TRY(wilson_apply_field(c, P64, X, 0, KX, 0, m));
  OVL_TRY(gram_host(c, X, 0, m, KX, 0, m, 0, H));
  std::vector<cd> C;
  if (kd_rayleigh_ritz_host(m, E, H, theta, C) != OVL_OK)
    return set_err(c, OVL_EBREAKDOWN, "kernel deflation: the filtered block lost linear independence");
  OVL_TRY(combine_host(c, X, 0, m, C, Xn, 0, m, 0));
  OVL_TRY(combine_host(c, KX, 0, m, C, KXn, 0, m, 0));
  std::vector<cd> one(m, 1.0), mt(m);
  for (int j = 0; j < m; ++j) mt[j] = -theta[j];
  OVL_TRY(axpby_batch(c, one, KXn, 0, mt, Xn, 0, R, 0, m));
  OVL_TRY(norms_batch(c, R, 0, m, res));
  OVL_TRY(norms_batch(c, KXn, 0, m, q));
  for (auto& x : q) x *= x;
  return OVL_OK;
}

// X <- T_d((2 K^2 - (b2 + c2)) / (b2 - c2)) X, the three-term Chebyshev recurrence on the block.
ovl_status kd_filter(ovl_ctx* c, Field*& X, Field*& Y1, Field*& Y2, Field& T, Field& K2, int m, int degree, double c2,
                     double b2) {
  const double e = 0.5 * (b2 - c2), cen = 0.5 * (b2 + c2);
  auto k2 = [&](Field& in, Field& out) -> ovl_status {
    OVL_TRY(wilson_apply_field(c, P64, in, 0, T, 0, m));
    return wilson_apply_field(c, P64, T, 0, out, 0, m);
  };
  // Y1 = (K^2 X - cen X) / e
  OVL_TRY(k2(*X, K2));
  std::vector<cd> a(m, 1.0 / e), b(m, -cen / e), one(m, 1.0), mone(m, -1.0), a2(m, 2.0 / e), b2v(m, -2.0 * cen / e);
  OVL_TRY(axpby_batch(c, a, K2, 0, b, *X, 0, *Y1, 0, m));
  for (int k = 2; k <= degree; ++k) {
    // Y2 = 2 (K^2 Y1 - cen Y1) / e - X
    OVL_TRY(k2(*Y1, K2));
    OVL_TRY(axpby_batch(c, a2, K2, 0, b2v, *Y1, 0, *Y2, 0, m));
    OVL_TRY(axpby_batch(c, one, *Y2, 0, mone, *X, 0, *Y2, 0, m));
    Field* t = X;
    X = Y1;
    Y1 = Y2;
    Y2 = t;
  }
  // the filtered block is Y1; rescale each vector to unit norm (the growth of T_d below c2)
  std::vector<double> nrm;
  OVL_TRY(norms_batch(c, *Y1, 0, m, nrm));
  std::vector<cd> s(m), z(m, 0.0);
  for (int j = 0; j < m; ++j) s[j] = nrm[j] > 0 ? 1.0 / nrm[j] : 1.0;
  OVL_TRY(axpby_batch(c, s, *Y1, 0, z, *Y1, 0, *X, 0, m));
  return OVL_OK;
}

}  // namespace
}  // namespace ovl

using namespace ovl;

extern "C" ovl_status ovl_host_rayleigh_ritz(int m, const double* E, const double* H, double* theta, double* C) {
  if (m < 1 || m > 1024 || !E || !H || !theta || !C) return OVL_EINVAL;
  const size_t mm = (size_t)m * m;
  for (size_t i = 0; i < 2 * mm; ++i)
    if (!std::isfinite(E[i]) || !std::isfinite(H[i])) return OVL_EINVAL;
  const cd* e = reinterpret_cast<const cd*>(E);
  const cd* h = reinterpret_cast<const cd*>(H);
  std::vector<double> th;
  std::vector<cd> c;
  const ovl_status st = kd_rayleigh_ritz_host(m, std::vector<cd>(e, e + mm), std::vector<cd>(h, h + mm), th, c);
  if (st != OVL_OK) return st;
  std::memcpy(theta, th.data(), sizeof(double) * m);
  std::memcpy(C, c.data(), sizeof(cd) * mm);
  return OVL_OK;
}

extern "C" ovl_status ovl_kernel_deflate(ovl_ctx* c, int n_ev, double tol, int max_iter, int n_poles, double* lambda,
                                         double* residual, double* a_out, int* n_poles_out, int* iters_done) {
  if (!c) return OVL_EINVAL;
  if (n_ev < 0 || n_ev > 256) return set_err(c, OVL_EINVAL, "n_ev must lie in 0..256");
  if (n_poles < 0 || n_poles > NPMAX) return set_err(c, OVL_EINVAL, "n_poles must be 0 (automatic) or lie in 1..64");
  // back to the full operator (a new deflation starts from it)
  if (c->kd_n > 0) {
    c->kd_n = 0;
    c->kd_lambda.clear();
    free_field(c->kd);
    OVL_TRY(set_poles(c, c->npoles0, c->za0, c->zb));
  }
  if (n_ev == 0) {
    if (a_out) *a_out = c->za;
    if (n_poles_out) *n_poles_out = c->npoles;
    if (iters_done) *iters_done = 0;
    return OVL_OK;
  }
  if (!(tol > 0) || max_iter < 1) return set_err(c, OVL_EINVAL, "need tol > 0 and max_iter >= 1");
  const int m = n_ev + std::max(8, n_ev);
  Field *X, *KX, *Y1, *Y2, *T, *K2, *R;
  OVL_TRY(get_field(c, "kd_X", P64, m, &X));
  OVL_TRY(get_field(c, "kd_KX", P64, m, &KX));
  OVL_TRY(get_field(c, "kd_Y1", P64, m, &Y1));
  OVL_TRY(get_field(c, "kd_Y2", P64, m, &Y2));
  OVL_TRY(get_field(c, "kd_T", P64, m, &T));
  OVL_TRY(get_field(c, "kd_K2", P64, m, &K2));
  OVL_TRY(get_field(c, "kd_R", P64, m, &R));
  // random start (fixed seed: the result does not depend on the call history)
  {
    std::mt19937_64 gen(0x5DEECE66DULL);
    std::normal_distribution<double> nd;
    std::vector<double> h((size_t)24 * c->V);
    for (int j = 0; j < m; ++j) {
      for (auto& x : h) x = nd(gen);
      OVL_TRY(import_spinors(c, h.data(), OVL_C128, 0, 1, *X, j));
    }
  }
  const double b2 = c->zb * c->zb;
  std::vector<double> theta, res, q;
  // first Rayleigh-Ritz on the random block, for the cut of the first filter
  OVL_TRY(kd_rayleigh_ritz(c, *X, *KX, *Y1, *K2, *R, m, theta, res, q));
  std::swap(X, Y1);
  int it = 0;
  bool conv = false;
  for (; it < max_iter && !conv; ++it) {
    // cut: the largest Rayleigh quotient of K^2 over the block (the signed Ritz values of
    // the indefinite K sit near zero for a block far from the low modes, so they cannot
    // serve); degree: at most 24 and such that the filter grows by at most 1e6 below the cut,
    // which keeps the block's Gram matrix well conditioned for the Cholesky of the next step
    double c2 = *std::max_element(q.begin(), q.end());
    c2 = std::min(c2, 0.5 * b2);
    const double smin = 0.5 * (b2 + c2) / (0.5 * (b2 - c2));
    const int degree = std::max(2, std::min(24, (int)std::floor(std::acosh(1e6) / std::acosh(smin))));
    OVL_TRY(kd_filter(c, X, Y1, Y2, *T, *K2, m, degree, c2, b2));
    OVL_TRY(kd_rayleigh_ritz(c, *X, *KX, *Y1, *K2, *R, m, theta, res, q));
    std::swap(X, Y1);
    conv = true;
    for (int i = 0; i < n_ev; ++i) conv = conv && res[i] <= tol;
  }
  if (!conv) {
    char msg[200];
    double worst = 0.0;
    for (int i = 0; i < n_ev; ++i) worst = std::max(worst, res[i]);
    snprintf(msg, sizeof(msg), "kernel deflation: %d of the lowest eigenpairs of K not within %.2e after %d "
             "iterations (worst residual %.3e)", n_ev, tol, it, worst);
    return set_err(c, OVL_ENOCONV, msg);
  }
  // keep the converged vectors
  Field kd;
  kd.prec = P64;
  kd.n = n_ev;
  kd.V = c->V;
  OVL_CUDA(c, cudaMalloc(&kd.data, kd.chunk_bytes()));
  c->kd = kd;
  {
    const ovl_status cs = copy_convert(c, *X, 0, c->kd, 0, n_ev);
    if (cs != OVL_OK) {
      free_field(c->kd);
      return cs;
    }
  }
  c->kd_lambda.assign(theta.begin(), theta.begin() + n_ev);
  c->kd_n = n_ev;
  // the interval left: lambda_min of K^2 on the complement
  double lmin, lmax;
  OVL_TRY(lanczos_bounds(c, 300, &lmin, &lmax, &c->kd, n_ev));
  // (the block's next Ritz value cannot bound it: the Ritz values of the indefinite K of
  // an unconverged vector may lie anywhere in its spectrum)
  double a = 0.95 * std::sqrt(std::max(lmin, 0.0));
  a = std::max(a, c->za0);
  int np = n_poles;
  if (np == 0) {
    for (np = 1; np < NPMAX; ++np) {
      std::vector<double> om(np), sg(np);
      double d = 0.0;
      if (zolotarev_coeffs(np, a, c->zb, om.data(), sg.data(), &d) == 0 && d <= c->eps_sign) break;
    }
  }
  ovl_status s = set_poles(c, np, a, c->zb);
  if (s != OVL_OK) {
    c->kd_n = 0;
    c->kd_lambda.clear();
    free_field(c->kd);
    set_poles(c, c->npoles0, c->za0, c->zb);
    return s;
  }
  if (lambda) memcpy(lambda, c->kd_lambda.data(), sizeof(double) * n_ev);
  if (residual) memcpy(residual, res.data(), sizeof(double) * n_ev);
  if (a_out) *a_out = a;
  if (n_poles_out) *n_poles_out = np;
  if (iters_done) *iters_done = it;
  return OVL_OK;
}
