// eigSUMR and eigCG accumulation (Sec. 5, Algs. 5-6). While the middle SUMR solve builds
// its Krylov basis, every step stores v_k = q_j and w_k = V q_j (V = gamma5 eps(K)),
// so that v^D_k = (1-mu)/2 w_k + (1+mu)/2 q_j = D q_j (Alg. 5). When k reaches the
// basis size m the Ritz recalculation of Alg. 6 runs:
//   E = (v_i, v_j), Cholesky E = U^dag U, M = (v^D_i, v^D_j) + 2 mu delta (v_i, gamma5 v^D_j),
//   eigenvectors Y of L^-1 M U^-1 (ascending), new v = V U^-1 Y, new v^D likewise,
//   keep the lowest n; residuals ||gamma5 v^D_i - v_i (v_i, gamma5 v^D_i)||.
// The Gram blocks run on the GPU (tensor cores with FP64-level accuracy by default, see
// tcgram.cu); the m x m algebra is FP64 on the host. If the basis has lost linear independence (Sec. 5 notes that
// orthogonality of the SUMR vectors is quickly lost with an inexact sign) and the
// Cholesky factor does not exist, or has a pivot below 1e-10 of the largest diagonal of E,
// the basis is orthonormalised through the eigendecomposition of E instead, dropping
// directions below 1e-10 of its largest eigenvalue.
//
// Sign accuracy while accumulating: the bound of Sec. 5.1 (the one used for the
// paper's runs),
//   ||delta^D|| < (chi sqrt(eps^2 + r0^2) - r0) / (sqrt((m-n) k) max |(UV)_ij|),
// chi = 1 for the first two diagonalisations and sqrt(n) after, r0 the residual of
// the best converged eigenvector, max |(UV)_ij| over the new basis vectors averaged
// over the last ten diagonalisations; the inversion relaxation is then capped by it
// (strategy 3 of Sec. 5.1: the more accurate of the two bounds).
#include <string.h>

#include <algorithm>
#include <cmath>

#include "context.h"
#include "eig.h"
#include "hostmath.h"
#include "solver.h"

namespace ovl {

// The k x k algebra of a Ritz step (Alg. 6), on the host in FP64, from the Gram blocks of a
// basis v_1 .. v_k with v^D_i = D v_i: E = (v_i, v_j), MVD = (v^D_i, v^D_j) and
// G5 = (v_i, gamma5 v^D_j), row-major. Gives the Ritz values (ascending), the coefficients C
// (k x keep, row-major) of the kept Ritz vectors in the basis, their residual norms
// ||gamma5 v^D - v (v, gamma5 v^D)||, and whether E had no Cholesky factor (the basis is then
// orthonormalised through the eigendecomposition of E, dropping directions below 1e-10 of
// its largest eigenvalue). restart: the locally optimal restart described in ritz_step.
void ritz_host(int k, const cd* E_in, const cd* MVD_in, const cd* G5_in, double mu, double delta, int keep,
               bool restart, RitzHost* out) {
  const size_t kk2 = (size_t)k * k;
  std::vector<cd> E(E_in, E_in + kk2);
  const std::vector<cd> MVD(MVD_in, MVD_in + kk2), G5(G5_in, G5_in + kk2);
  keep = std::min(keep, k);
  out->cholesky_fallback = false;
  std::vector<cd> M((size_t)k * k);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) M[(size_t)i * k + j] = MVD[(size_t)i * k + j] + 2.0 * mu * delta * G5[(size_t)i * k + j];
  for (int i = 0; i < k; ++i)
    for (int j = i; j < k; ++j) {
      const cd h = 0.5 * (M[(size_t)i * k + j] + std::conj(M[(size_t)j * k + i]));
      M[(size_t)i * k + j] = h;
      M[(size_t)j * k + i] = std::conj(h);
      const cd g = 0.5 * (E[(size_t)i * k + j] + std::conj(E[(size_t)j * k + i]));
      E[(size_t)i * k + j] = g;
      E[(size_t)j * k + i] = std::conj(g);
    }
  // B: k x r with B^dag E B = 1
  std::vector<cd> B;
  int r = k;
  {
    // the Cholesky coordinates only while every pivot L_jj^2 stays above 1e-10 of the largest
    // diagonal of E (the cut the eigendecomposition below applies to E's eigenvalues): a
    // nearly dependent basis (SUMR vectors lose orthogonality with an inexact sign, Sec. 5)
    // can pass the factorisation with a pivot at rounding level, and U^-1 ~ 1/pivot then
    // wrecks the projected matrix
    std::vector<cd> L = E;
    double emax = 0.0;
    for (int i = 0; i < k; ++i) emax = std::max(emax, E[(size_t)i * k + i].real());
    bool chol = cholesky_lower(k, L.data()) == 0;
    for (int i = 0; chol && i < k; ++i) chol = std::norm(L[(size_t)i * k + i]) >= 1e-10 * emax;
    if (chol) {
      std::vector<cd> Li((size_t)k * k);
      lower_inverse(k, L.data(), Li.data());
      B.resize((size_t)k * k);
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) B[(size_t)i * k + j] = std::conj(Li[(size_t)j * k + i]);   // L^-dag = U^-1
    } else {
      std::vector<cd> Ec = E, Z((size_t)k * k);
      std::vector<double> w(k);
      eigh_herm(k, Ec.data(), w.data(), Z.data());
      const double thr = 1e-10 * std::max(w[k - 1], 1e-300);
      std::vector<int> keepc;
      for (int i = 0; i < k; ++i)
        if (w[i] > thr) keepc.push_back(i);
      r = (int)keepc.size();
      B.assign((size_t)k * r, 0.0);
      for (int i = 0; i < k; ++i)
        for (int jj = 0; jj < r; ++jj) B[(size_t)i * r + jj] = Z[(size_t)i * k + keepc[jj]] / std::sqrt(w[keepc[jj]]);
      out->cholesky_fallback = true;
    }
  }
  // T = B^dag M B (r x r)
  std::vector<cd> MB((size_t)k * r), T((size_t)r * r), Y((size_t)r * r);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < r; ++j) {
      cd s = 0;
      for (int l = 0; l < k; ++l) s += M[(size_t)i * k + l] * B[(size_t)l * r + j];
      MB[(size_t)i * r + j] = s;
    }
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) {
      cd s = 0;
      for (int l = 0; l < k; ++l) s += std::conj(B[(size_t)l * r + i]) * MB[(size_t)l * r + j];
      T[(size_t)i * r + j] = s;
    }
  std::vector<double> lam(r);
  std::vector<cd> T0 = T;
  eigh_herm(r, T.data(), lam.data(), Y.data());
  keep = std::min(keep, r);
  // Locally optimal restart (the eigCG restart that the accumulation of Sec. 5 adapts):
  // at a basis restart keep the lowest Ritz vectors of the whole basis and those of the
  // basis without its newest vector, Rayleigh-Ritz on their span. With the Cholesky
  // coordinates (B upper triangular) the first k-1 columns of B span the first k-1
  // basis vectors, so the second set comes from the leading block of T.
  const bool lo = restart && r == k && 2 * keep + 1 <= k;
  int nout = keep;
  std::vector<cd> Yc((size_t)r * keep);   // r x nout coefficients in B coordinates
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < keep; ++j) Yc[(size_t)i * keep + j] = Y[(size_t)i * r + j];
  if (lo) {
    const int k1 = k - 1;
    std::vector<cd> T1((size_t)k1 * k1), Y1((size_t)k1 * k1);
    for (int i = 0; i < k1; ++i)
      for (int j = 0; j < k1; ++j) T1[(size_t)i * k1 + j] = T0[(size_t)i * k + j];
    std::vector<double> lam1(k1);
    eigh_herm(k1, T1.data(), lam1.data(), Y1.data());
    // Z = [Y[:, :keep], (Y1[:, :keep]; 0)], orthonormalised (modified Gram-Schmidt)
    std::vector<std::vector<cd>> Z;
    for (int j = 0; j < 2 * keep; ++j) {
      std::vector<cd> z(k, 0.0);
      if (j < keep)
        for (int i = 0; i < k; ++i) z[i] = Y[(size_t)i * k + j];
      else
        for (int i = 0; i < k1; ++i) z[i] = Y1[(size_t)i * k1 + (j - keep)];
      for (int pass = 0; pass < 2; ++pass)
        for (const auto& q : Z) {
          cd d = 0;
          for (int i = 0; i < k; ++i) d += std::conj(q[i]) * z[i];
          for (int i = 0; i < k; ++i) z[i] -= d * q[i];
        }
      double nz = 0;
      for (int i = 0; i < k; ++i) nz += std::norm(z[i]);
      nz = std::sqrt(nz);
      if (nz < 1e-8) continue;
      for (int i = 0; i < k; ++i) z[i] /= nz;
      Z.push_back(z);
    }
    const int q = (int)Z.size();
    // Rayleigh-Ritz on span Z: T2 = Z^dag T Z, with T Z formed once (k^2 q + q^2 k
    // products instead of q^2 k^2; the same sums in the same order)
    std::vector<cd> T2((size_t)q * q), Y2((size_t)q * q), TZ((size_t)k * q);
    for (int b2 = 0; b2 < q; ++b2)
      for (int i = 0; i < k; ++i) {
        cd ti = 0;
        for (int l = 0; l < k; ++l) ti += T0[(size_t)i * k + l] * Z[b2][l];
        TZ[(size_t)i * q + b2] = ti;
      }
    for (int a2 = 0; a2 < q; ++a2)
      for (int b2 = 0; b2 < q; ++b2) {
        cd sacc = 0;
        for (int i = 0; i < k; ++i) sacc += std::conj(Z[a2][i]) * TZ[(size_t)i * q + b2];
        T2[(size_t)a2 * q + b2] = sacc;
      }
    for (int a2 = 0; a2 < q; ++a2)
      for (int b2 = a2 + 1; b2 < q; ++b2) {
        const cd h = 0.5 * (T2[(size_t)a2 * q + b2] + std::conj(T2[(size_t)b2 * q + a2]));
        T2[(size_t)a2 * q + b2] = h;
        T2[(size_t)b2 * q + a2] = std::conj(h);
      }
    std::vector<double> lam2(q);
    eigh_herm(q, T2.data(), lam2.data(), Y2.data());
    nout = q;
    Yc.assign((size_t)r * nout, 0.0);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < nout; ++j) {
        cd sacc = 0;
        for (int l = 0; l < q; ++l) sacc += Z[l][i] * Y2[(size_t)l * q + j];
        Yc[(size_t)i * nout + j] = sacc;
      }
    lam.assign(lam2.begin(), lam2.end());
  }
  keep = nout;
  // C = B Yc  (k x keep)
  std::vector<cd> C((size_t)k * keep);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < keep; ++j) {
      cd s = 0;
      for (int l = 0; l < r; ++l) s += B[(size_t)i * r + l] * Yc[(size_t)l * keep + j];
      C[(size_t)i * keep + j] = s;
    }
  // Ritz values and residuals from the Gram data: ||r||^2 = ||v^D||^2 - |(v, g5 v^D)|^2
  out->lam.assign(lam.begin(), lam.begin() + keep);
  out->res.assign(keep, 0.0);
  for (int j = 0; j < keep; ++j) {
    cd nd = 0, th = 0;
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q) {
        const cd w = std::conj(C[(size_t)p * keep + j]) * C[(size_t)q * keep + j];
        nd += w * MVD[(size_t)p * k + q];
        th += w * G5[(size_t)p * k + q];
      }
    out->res[j] = std::sqrt(std::max(0.0, nd.real() - std::norm(th)));
  }
  out->C = C;
  out->keep = keep;
}

ovl_status ritz_step(ovl_ctx* c, EigState* e, int keep, bool restart) {
  const int k = e->k;
  if (k == 0) return OVL_OK;
  keep = std::min(keep, k);
  const double mu = e->mu, delta = e->delta;
  const double a = 0.5 * (1.0 - mu), b = 0.5 * (1.0 + mu);
  Field* VD;
  OVL_TRY(get_field(c, "e_VD", e->prec, e->m, &VD));
  {
    std::vector<cd> aa(k, a), bb(k, b);
    OVL_TRY(axpby_batch(c, aa, *e->W, 0, bb, *e->V, 0, *VD, 0, k));
  }
  std::vector<cd> E, MVD, G5;
  OVL_TRY(gram_host(c, *e->V, 0, k, *e->V, 0, k, 0, E));
  OVL_TRY(gram_host(c, *VD, 0, k, *VD, 0, k, 0, MVD));
  OVL_TRY(gram_host(c, *e->V, 0, k, *VD, 0, k, 1, G5));
  RitzHost rh;
  ritz_host(k, E.data(), MVD.data(), G5.data(), mu, delta, keep, restart, &rh);
  if (rh.cholesky_fallback) e->cholesky_fallbacks += 1;
  keep = rh.keep;
  const std::vector<cd>& C = rh.C;
  // rotate v and w
  Field* Tv;
  OVL_TRY(get_field(c, "e_T", e->prec, e->m, &Tv));
  OVL_TRY(combine_host(c, *e->V, 0, k, C, *Tv, 0, keep, 0));
  OVL_TRY(copy_convert(c, *Tv, 0, *e->V, 0, keep));
  OVL_TRY(combine_host(c, *e->W, 0, k, C, *Tv, 0, keep, 0));
  OVL_TRY(copy_convert(c, *Tv, 0, *e->W, 0, keep));
  e->ritz = rh.lam;
  e->res = rh.res;
  // largest coefficient of the newly added vectors in the kept eigenvectors
  double mx = 0.0;
  for (int p = e->n_seeded; p < k; ++p)
    for (int j = 0; j < keep; ++j) mx = std::max(mx, std::abs(C[(size_t)p * keep + j]));
  e->uv_hist.push_back(mx);
  if (e->uv_hist.size() > 10) e->uv_hist.erase(e->uv_hist.begin());
  e->ndiag += 1;
  e->k = keep;
  e->n_seeded = keep;
  // next sign-accuracy cap (Sec. 5.1 bound)
  double avg = 0.0;
  for (double v : e->uv_hist) avg += v;
  avg /= std::max<size_t>(1, e->uv_hist.size());
  const double r0 = *std::min_element(e->res.begin(), e->res.end());
  const double chi = e->ndiag <= 2 ? 1.0 : std::sqrt((double)e->n_eig);
  const double num = chi * std::sqrt(e->eps_v * e->eps_v + r0 * r0) - r0;
  const double den = std::sqrt((double)std::max(1, e->m - e->n_eig) * e->kk) * std::max(avg, 1e-12);
  double cap = num / den;
  if (!(cap > 0)) cap = e->eps_v;
  // The bound is absolute, but an error in v^D = D v only leaves the low Ritz pairs
  // usable while it is small against their singular values (Sec. 5.1 warns that too
  // low an accuracy for v^D makes the eigenvalue estimates diverge): cap it at 5% of
  // the smallest Ritz singular value (never below mu, the bound of D's spectrum).
  const double lmin = std::max(e->ritz.empty() ? mu * mu : e->ritz[0], mu * mu);
  cap = std::min(cap, 0.05 * std::sqrt(lmin));
  e->eta_cap = std::min(std::max(cap, 1e-10), c->P.eta_floor);
  if (e->eig) e->eig->eta_cap = e->eta_cap;
  return OVL_OK;
}

// eigCG (Sec. 5): system 0's residual directions of the middle relCG solve feed the basis.
// v = (t_j - beta_{j-1} t_{j-1}) / ||r_j|| is Hhat^-1 r_j (r_j the CG residual; with no
// deflation Hhat = 1 and these are the Lanczos vectors of H^2), and its
// v^D = D v = gamma5 (z_j - beta_{j-1} z_{j-1}) / ||r_j||; the basis keeps
// w = gamma5 eps(K) v = (2 v^D - (1+mu) v) / (1-mu), the form the Ritz step and the
// deflation space use (D v = (1+mu)/2 v + (1-mu)/2 w).
ovl_status eig_cg_hook(ovl_ctx* c, void* data, const Field& t, const Field& z,
                       const std::vector<std::complex<double>>& beta_prev, const std::vector<double>& rnorm,
                       int iter) {
  EigState* e = static_cast<EigState*>(data);
  const double rn = rnorm.empty() ? 0.0 : rnorm[0];
  if (!(rn > 0.0) || !std::isfinite(rn)) return OVL_OK;
  const double mu = e->mu;
  const cd bp = iter > 0 ? beta_prev[0] : cd(0.0);
  const cd inv = 1.0 / rn;
  Field* tmp;
  OVL_TRY(get_field(c, "e_tmp", e->prec, 1, &tmp));
  // v = (t - bp t_prev) / ||r||
  std::vector<cd> a1(1, inv), b1(1, -bp * inv), zero(1, 0.0);
  if (iter > 0) {
    OVL_TRY(axpby_batch(c, a1, t, 0, b1, *e->Tprev, 0, *e->V, e->k, 1));
  } else {
    OVL_TRY(axpby_batch(c, a1, t, 0, zero, t, 0, *e->V, e->k, 1));
  }
  // v^D = gamma5 (z - bp z_prev) / ||r||, then w = (2 v^D - (1+mu) v) / (1-mu)
  if (iter > 0) {
    OVL_TRY(axpby_batch(c, a1, z, 0, b1, *e->Zprev, 0, *tmp, 0, 1));
  } else {
    OVL_TRY(axpby_batch(c, a1, z, 0, zero, z, 0, *tmp, 0, 1));
  }
  launch_gamma5(e->prec, tmp->ref(), 1, c->V, c->st);
  std::vector<cd> a2(1, 2.0 / (1.0 - mu)), b2(1, -(1.0 + mu) / (1.0 - mu));
  OVL_TRY(axpby_batch(c, a2, *tmp, 0, b2, *e->V, e->k, *e->W, e->k, 1));
  OVL_TRY(copy_convert(c, t, 0, *e->Tprev, 0, 1));
  OVL_TRY(copy_convert(c, z, 0, *e->Zprev, 0, 1));
  e->k += 1;
  if (e->k == e->m) OVL_TRY(ritz_step(c, e, e->n_eig, true));
  return OVL_OK;
}

ovl_status eig_hook(ovl_ctx* c, void* data, const Field& q, const Field& u, int iter) {
  (void)iter;
  EigState* e = static_cast<EigState*>(data);
  // system 0 of the batch feeds the basis
  OVL_TRY(copy_convert(c, q, 0, *e->V, e->k, 1));
  OVL_TRY(copy_convert(c, u, 0, *e->W, e->k, 1));
  e->k += 1;
  if (e->k == e->m) OVL_TRY(ritz_step(c, e, e->n_eig, true));
  return OVL_OK;
}

}  // namespace ovl
