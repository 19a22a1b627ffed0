// Solvers of liboverlap (host control, device vectors), all on lock-step batches
// of independent systems D(mu_j) x_j = b_j:
//
//  * relSUMR (Secs. 2-3) on A = rho + V, V = gamma5 eps(K), rho = (1+mu)/(1-mu), so
//    D = (1-mu)/2 A. The Krylov basis is Alg. 1 (q, q~, gamma_j, sigma_j). The printed
//    Alg. 2 leaves zeta undefined and, under every reading tried, does not reproduce
//    the minimal-residual iterates, so the update is re-derived from App. A: a
//    progressive Givens QR of rho I^ + B^ whose rows above the subdiagonal are
//    gamma_j times the coefficients of q~_j, which gives short recurrences with two
//    auxiliary vectors (p, S). In exact arithmetic the iterates equal GMRES's.
//    Relaxation eta_j = eps_A ||b|| / ||r_j||, never worse than the floor (Sec. 3).
//  * relCG (Sec. 3) as the spectrally preconditioned CGNE of Alg. 4 on H^2, H =
//    gamma5 D, with eta_j = eps_A ||b|| sqrt(zeta), zeta = sum_i ||r_i||^-2.
//  * GMRESR (Alg. 3) in FP64 around either, with c = A u at accuracy
//    eps ||b|| / ||r|| relative to ||u||.
//  * eigSUMR (Algs. 5-6) and the deflated starts of Sec. 4.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>

#include "context.h"
#include "hostmath.h"
#include "solver.h"

namespace ovl {

// OVL_LOG=1 in the environment prints one line per outer step and per middle-solve step.
static int log_level() {
  static int lv = -1;
  if (lv < 0) {
    const char* e = getenv("OVL_LOG");
    lv = e ? atoi(e) : 0;
  }
  return lv;
}

// ------------------------------------------------------------------ helpers
ovl_status dots_batch(ovl_ctx* c, const Field& x, int xoff, const Field& y, int yoff, int n, std::vector<cd>& out) {
  OVL_TRY(ensure_partials(c, n));
  launch_dot(x.prec, x.ref(xoff), y.prec, y.ref(yoff), n, c->V, c->partials, c->st);
  std::vector<double> h(2 * n);
  OVL_TRY(reduce_to_host(c, make_shape(c->V, n).nsb, n, h.data()));
  out.resize(n);
  for (int j = 0; j < n; ++j) out[j] = cd(h[2 * j], h[2 * j + 1]);
  return OVL_OK;
}

ovl_status norms_batch(ovl_ctx* c, const Field& x, int xoff, int n, std::vector<double>& out) {
  OVL_TRY(ensure_partials(c, n));
  launch_norm2(x.prec, x.ref(xoff), n, c->V, c->partials, c->st);
  std::vector<double> h(2 * n);
  OVL_TRY(reduce_to_host(c, make_shape(c->V, n).nsb, n, h.data()));
  out.resize(n);
  // a NaN stays NaN (std::max(0.0, NaN) would be 0, a "perfect" norm)
  for (int j = 0; j < n; ++j) out[j] = std::isnan(h[2 * j]) ? h[2 * j] : std::sqrt(std::max(0.0, h[2 * j]));
  return OVL_OK;
}

// z = a x + b y with per-system complex a, b (z may alias x or y; all same precision)
ovl_status axpby_batch(ovl_ctx* c, const std::vector<cd>& a, const Field& x, int xoff, const std::vector<cd>& b,
                       const Field& y, int yoff, Field& z, int zoff, int n) {
  std::vector<double> h(4 * n);
  for (int j = 0; j < n; ++j) {
    h[2 * j] = a[j].real();
    h[2 * j + 1] = a[j].imag();
    h[2 * n + 2 * j] = b[j].real();
    h[2 * n + 2 * j + 1] = b[j].imag();
  }
  const double* d;
  OVL_TRY(upload(c, h.data(), 4 * n, &d));
  launch_axpby(z.prec, d, d + 2 * n, x.ref(xoff), y.ref(yoff), z.ref(zoff), n, c->V, c->st);
  OVL_TRY(check_launch(c, __func__));
  return OVL_OK;
}

ovl_status copy_convert(ovl_ctx* c, const Field& in, int ioff, Field& out, int ooff, int n) {
  if (in.prec == out.prec) {
    const size_t per = (size_t)c->V * spinor_site_bytes(in.prec);
    OVL_CUDA(c, cudaMemcpyAsync((char*)out.data + per * ooff, (char*)in.data + per * ioff, per * n,
                                cudaMemcpyDeviceToDevice, c->st));
    if (in.prec == P16)
      OVL_CUDA(c, cudaMemcpyAsync(out.norm + (size_t)c->V * ooff, in.norm + (size_t)c->V * ioff,
                                  sizeof(float) * c->V * n, cudaMemcpyDeviceToDevice, c->st));
    return OVL_OK;
  }
  launch_convert(in.prec, in.ref(ioff), out.prec, out.ref(ooff), n, c->V, c->st);
  OVL_TRY(check_launch(c, __func__));
  return OVL_OK;
}

// Gram block G = (A_i, [g5] B_j), na x nb complex row-major, into dG (the last 2 na nb
// doubles of the work buffer, returned): launched on the context stream, not waited for.
// *derr is the tensor-core path's device error flag (nullptr on the CUDA-core path).
ovl_status gram_device(ovl_ctx* c, const Field& A, int aoff, int na, const Field& B, int boff, int nb, int g5,
                       double** dGout, int** derr) {
  const size_t gsz = (size_t)na * nb * 2;
  const bool tc = c->P.gram_method == 0 && tc_gram_supported(A.prec, B.prec);
  int nsplit = 0;
  size_t need = gsz * 1300 + gsz;
  if (tc) {
    int nsm = 0;
    OVL_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    nsplit = tc_gram_splits(na, nb, c->V, nsm);
    // partials, then na + nb exponents and the error flag (as ints), then G
    need = tc_gram_work_doubles(na, nb, nsplit) + (size_t)(na + nb + 2) / 2 + 1 + gsz;
  }
  OVL_TRY(ensure_work(c, need));
  double* dG = c->dwork + c->dwork_n - gsz;
  OVL_CUDA(c, cudaMemsetAsync(dG, 0, gsz * sizeof(double), c->st));
  *derr = nullptr;
  ProfPair pp;
  prof_begin(c, 6, &pp);
  if (tc) {
    const size_t nw = tc_gram_work_doubles(na, nb, nsplit);
    int* ex = reinterpret_cast<int*>(c->dwork + nw);
    *derr = ex + na + nb;
    OVL_CUDA(c, cudaMemsetAsync(*derr, 0, sizeof(int), c->st));
    launch_tc_gram(A.prec, A.ref(aoff).data, na, B.prec, B.ref(boff).data, nb, c->V, g5, nsplit, dG, c->dwork, ex,
                   *derr, c->st);
  } else {
    launch_gram(A.prec, A.ref(aoff), na, B.prec, B.ref(boff), nb, c->V, dG, c->dwork, c->dwork_n - gsz, g5, c->st);
  }
  prof_end(c, &pp, (double)c->V * ((double)na * spinor_site_bytes(A.prec) + (double)nb * spinor_site_bytes(B.prec)));
  OVL_TRY(check_launch(c, __func__));
  *dGout = dG;
  return OVL_OK;
}

// Gram block G = (A_i, [g5] B_j), na x nb, to the host (complex row-major).
ovl_status gram_host(ovl_ctx* c, const Field& A, int aoff, int na, const Field& B, int boff, int nb, int g5,
                     std::vector<cd>& G) {
  const size_t gsz = (size_t)na * nb * 2;
  double* dG = nullptr;
  int* derr = nullptr;
  OVL_TRY(gram_device(c, A, aoff, na, B, boff, nb, g5, &dG, &derr));
  int herr = 0;
  std::vector<double> h(gsz);
  OVL_CUDA(c, cudaMemcpyAsync(h.data(), dG, gsz * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if (derr) OVL_CUDA(c, cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  if (herr) return set_err(c, OVL_ETIMEOUT, "tensor-core Gram block: a bounded wait on the MMA pipeline gave up");
  G.resize((size_t)na * nb);
  for (size_t k = 0; k < G.size(); ++k) G[k] = cd(h[2 * k], h[2 * k + 1]);
  return OVL_OK;
}

// Y_j (+)= sum_i A_i C[i][j]
ovl_status combine_host(ovl_ctx* c, const Field& A, int aoff, int na, const std::vector<cd>& C, Field& Y, int yoff,
                        int ny, int add) {
  std::vector<double> h((size_t)na * ny * 2);
  for (size_t k = 0; k < (size_t)na * ny; ++k) {
    h[2 * k] = C[k].real();
    h[2 * k + 1] = C[k].imag();
  }
  const double* d;
  OVL_TRY(upload(c, h.data(), (int)h.size(), &d));
  ProfPair pp;
  prof_begin(c, 6, &pp);
  launch_combine(A.prec, A.ref(aoff), na, d, Y.prec, Y.ref(yoff), ny, c->V, add, c->st);
  prof_end(c, &pp, (double)c->V * ((double)na * spinor_site_bytes(A.prec) + (double)ny * (add + 1) * spinor_site_bytes(Y.prec)));
  OVL_TRY(check_launch(c, __func__));
  return OVL_OK;
}

// ------------------------------------------------------------------ overlap apply
// out_j = D(mu_j) v_j (herm: gamma5 D(mu_j) v_j) at sign accuracy eta_j.
ovl_status overlap_apply_batch(ovl_ctx* c, const Field& v, int voff, Field& out, int ooff, int n,
                               const std::vector<double>& mus, const std::vector<double>& eta, int herm, int mode,
                               long long* wcalls_out) {
  std::vector<double> coef(2 * n);
  for (int j = 0; j < n; ++j) {
    coef[2 * j] = 0.5 * (1.0 + mus[j]);
    coef[2 * j + 1] = 0.5 * (1.0 - mus[j]);
  }
  double emin = 1e300;
  for (double e : eta) emin = std::min(emin, e > 0 ? e : c->eps_sign);
  if (mode < 0) mode = choose_mode(c, emin);
  SignStats ss;
  OVL_TRY(sign_op(c, mode, v, voff, out, ooff, n, eta.data(), 0, 0, coef.data(), herm, nullptr, 0, nullptr, &ss));
  if (wcalls_out) {
    for (int j = 0; j < n; ++j) wcalls_out[j] += (long long)(2 * ss.iters[j] + 1) * (mode == SIGN64 || mode == SIGN64E ? 2 : 1);
  }
  return OVL_OK;
}

// ------------------------------------------------------------------ deflation data
// With psi_i (v) and w_i = gamma5 eps(K) psi_i held, D(mu) psi = (1+mu)/2 psi + (1-mu)/2 w.
ovl_status defl_prepare(ovl_ctx* c, ovl_defl* d) {
  if (d->prepared) return OVL_OK;
  const int n = d->n;
  OVL_TRY(gram_host(c, d->v, 0, n, d->v, 0, n, 0, d->VV));
  OVL_TRY(gram_host(c, d->w, 0, n, d->w, 0, n, 0, d->WW));
  OVL_TRY(gram_host(c, d->w, 0, n, d->v, 0, n, 0, d->WV));
  OVL_TRY(gram_host(c, d->v, 0, n, d->v, 0, n, 1, d->G5VV));
  OVL_TRY(gram_host(c, d->v, 0, n, d->w, 0, n, 1, d->G5VW));
  d->prepared = true;
  return OVL_OK;
}

// (D psi)^dag (D psi) at mass mu, n x n, from the Gram blocks of psi and w
static void dd_matrix(int n, const cd* VV, const cd* WW, const cd* WV, double mu, std::vector<cd>& M) {
  const double a = 0.5 * (1.0 - mu), b = 0.5 * (1.0 + mu);
  M.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const cd wv = WV[(size_t)i * n + j];
      const cd vw = std::conj(WV[(size_t)j * n + i]);
      M[(size_t)i * n + j] = a * a * WW[(size_t)i * n + j] + a * b * (wv + vw) + b * b * VV[(size_t)i * n + j];
    }
}

// Sec. 4, SUMR variant, on the host: x0 = sum_j alpha_j psi'_j minimising ||b - D x0|| with
// psi' the rotation that diagonalises (psi_i, gamma5 D psi_j), from the Gram blocks of the
// space (n x n, row-major: VV = (psi_i, psi_j), WW = (w_i, w_j), WV = (w_i, psi_j),
// G5VV = (psi_i, gamma5 psi_j), G5VW = (psi_i, gamma5 w_j); D psi = (1+mu)/2 psi + (1-mu)/2 w)
// and, per system j, VB = (psi_l, b_j), WB = (w_l, b_j) (n x nsys). coefs (n x nsys): x0 on
// psi with the rotation folded in. per_vector: the per-vector alpha_j of Sec. 4 instead of
// the least-squares solve. OVL_EBREAKDOWN when the normal equations are singular.
ovl_status defl_start_host(int n, const cd* VV, const cd* WW, const cd* WV, const cd* G5VV, const cd* G5VW,
                           int nsys, const cd* VB, const cd* WB, const double* mus, bool per_vector, cd* coefs) {
  for (size_t i = 0; i < (size_t)n * nsys; ++i) coefs[i] = 0.0;
  // the rotation Y and the rotated normal matrix depend on the mass only: built once per
  // distinct mass of the batch (sources x masses share them)
  struct PerMass {
    double mu;
    std::vector<cd> Y, G;
  };
  std::vector<PerMass> per_mass;
  for (int j = 0; j < nsys; ++j) {
    const double mu = mus[j];
    const double a = 0.5 * (1.0 - mu), bb = 0.5 * (1.0 + mu);
    const PerMass* pm = nullptr;
    for (const auto& q : per_mass)
      if (q.mu == mu) pm = &q;
    if (pm == nullptr) {
      PerMass q;
      q.mu = mu;
      // Hs = (psi_i, gamma5 D psi_j) = b (psi, g5 psi) + a (psi, g5 w)
      std::vector<cd> Hs((size_t)n * n);
      std::vector<double> w(n);
      q.Y.resize((size_t)n * n);
      for (size_t k = 0; k < Hs.size(); ++k) Hs[k] = bb * G5VV[k] + a * G5VW[k];
      for (int i = 0; i < n; ++i)
        for (int k = i + 1; k < n; ++k) {
          const cd h = 0.5 * (Hs[(size_t)i * n + k] + std::conj(Hs[(size_t)k * n + i]));
          Hs[(size_t)i * n + k] = h;
          Hs[(size_t)k * n + i] = std::conj(h);
        }
      eigh_herm(n, Hs.data(), w.data(), q.Y.data());
      std::vector<cd> M;
      dd_matrix(n, VV, WW, WV, mu, M);
      // rotated normal equations: (Y^dag M Y) alpha = Y^dag (D psi)^dag b
      std::vector<cd> MY((size_t)n * n);
      q.G.resize((size_t)n * n);
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
          cd s = 0;
          for (int l = 0; l < n; ++l) s += M[(size_t)i * n + l] * q.Y[(size_t)l * n + k];
          MY[(size_t)i * n + k] = s;
        }
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
          cd s = 0;
          for (int l = 0; l < n; ++l) s += std::conj(q.Y[(size_t)l * n + i]) * MY[(size_t)l * n + k];
          q.G[(size_t)i * n + k] = s;
        }
      per_mass.push_back(std::move(q));
      pm = &per_mass.back();
    }
    const std::vector<cd>& Y = pm->Y;
    std::vector<cd> G = pm->G, rhs(n);   // lu_solve overwrites its matrix
    for (int i = 0; i < n; ++i) {
      cd s = 0;
      for (int l = 0; l < n; ++l) {
        const cd dpb = a * WB[(size_t)l * nsys + j] + bb * VB[(size_t)l * nsys + j];   // ((D psi_l), b)
        s += std::conj(Y[(size_t)l * n + i]) * dpb;
      }
      rhs[i] = s;
    }
    if (per_vector) {
      for (int i = 0; i < n; ++i) rhs[i] /= G[(size_t)i * n + i];
    } else if (lu_solve(n, G.data(), rhs.data(), 1) != 0) {
      return OVL_EBREAKDOWN;
    }
    for (int i = 0; i < n; ++i) {
      cd s = 0;
      for (int k = 0; k < n; ++k) s += Y[(size_t)i * n + k] * rhs[k];
      coefs[(size_t)i * nsys + j] = s;
    }
  }
  return OVL_OK;
}

// The deflated start of Sec. 4 for nsys systems: Gram blocks on the device, then
// defl_start_host. coefs (n_ev x nsys, column j) are x0 of system j on psi.
ovl_status defl_start(ovl_ctx* c, ovl_defl* d, const Field& b, int boff, int nsys, const std::vector<double>& mus,
                      std::vector<cd>& coefs) {
  OVL_TRY(defl_prepare(c, d));
  const int n = d->n;
  std::vector<cd> VB, WB;
  OVL_TRY(gram_host(c, d->v, 0, n, b, boff, nsys, 0, VB));
  OVL_TRY(gram_host(c, d->w, 0, n, b, boff, nsys, 0, WB));
  coefs.assign((size_t)n * nsys, 0.0);
  if (defl_start_host(n, d->VV.data(), d->WW.data(), d->WV.data(), d->G5VV.data(), d->G5VW.data(), nsys, VB.data(),
                      WB.data(), mus.data(), d->per_vector, coefs.data()) != OVL_OK)
    return set_err(c, OVL_EBREAKDOWN, "singular deflation normal equations");
  return OVL_OK;
}

// ------------------------------------------------------------------ SUMR recurrence
// Alg. 1 with the sign applied inexactly: gamma_j is the projection coefficient of u = V q_j
// on q~_j and sigma_j = ||u + gamma_j q~_j||, so that V q_j = sigma_j q_{j+1} - gamma_j q~_j
// holds for the computed vectors; with an exact (unitary) sign this is gamma_j = -(q~_j, u)
// and sigma_j = sqrt(1 - |gamma_j|^2) of Alg. 1. Inputs (q~, u), ||u||^2, ||q~||^2; false
// when the Krylov space is exhausted or the sign was not finite.
bool sumr_basis_step(cd qtu, double uu, double tt, cd* gam_out, double* sig_out) {
  const cd gam = tt > 0 ? -qtu / tt : cd(0.0);
  const double s2 = uu - std::norm(qtu) / std::max(tt, 1e-300);
  if (!(s2 > 1e-24 * std::max(uu, 1e-300)) || !std::isfinite(s2)) return false;
  *gam_out = gam;
  *sig_out = std::sqrt(s2);
  return true;
}

// One step of the short recurrence of one system (reading 7: the progressive Givens QR of
// rho I + B^, re-derived from App. A; its upper part is gamma_j times the coefficients of
// q~_j, carried by the two auxiliary vectors p and S). vals = {R_{j-1,j}, gamma_j
// sigma_{j-1}, 1/R_jj, sigma_{j-1}, zeta_{j-1}, g_j}: the coefficients of the vector update;
// s.ghat becomes the residual estimate after this step.
void sumr_rec_step(SumrRec& s, double rho, cd gam, double sig, cd vals[6]) {
  cd a, Rm1, zm1;
  if (s.it == 0) {
    s.zeta = 1.0;
    a = rho - gam * s.zeta;
    Rm1 = 0.0;
    zm1 = 0.0;
  } else {
    zm1 = s.cprev * s.sigprev * s.zeta + std::conj(s.sprev) * std::conj(s.gprev);
    s.zeta = -s.sprev * s.sigprev * s.zeta + s.cprev * std::conj(s.gprev);
    Rm1 = rho * std::conj(s.sprev) - gam * zm1;
    a = rho * s.cprev - gam * s.zeta;
  }
  const double nrm = std::sqrt(std::norm(a) + sig * sig);
  const double cc = std::abs(a) / nrm;
  const cd ss_ = std::abs(a) > 0 ? cc * sig / a : cd(1.0, 0.0);
  const cd Rjj = cc * a + std::conj(ss_) * sig;
  const cd g = cc * s.ghat;
  s.ghat = -ss_ * s.ghat;
  vals[0] = Rm1;
  vals[1] = gam * s.sigprev;
  vals[2] = 1.0 / Rjj;
  vals[3] = s.sigprev;
  vals[4] = zm1;
  vals[5] = g;
  s.cprev = cc;
  s.sprev = ss_;
  s.sigprev = sig;
  s.gprev = gam;
  s.it += 1;
}

// ------------------------------------------------------------------ relSUMR
ovl_status sumr_batch(ovl_ctx* c, const SumrCfg& cfg, int n, const std::vector<double>& mus, const Field& b, int boff,
                      Field& x, int xoff, SumrResult& res) {
  const int PS = cfg.prec;
  const int V = c->V;
  Field *fq, *fqt, *fp, *fS, *fu;
  OVL_TRY(get_field(c, "s_q", PS, n, &fq));
  OVL_TRY(get_field(c, "s_qt", PS, n, &fqt));
  OVL_TRY(get_field(c, "s_p", PS, n, &fp));
  OVL_TRY(get_field(c, "s_S", PS, n, &fS));
  OVL_TRY(get_field(c, "s_u", PS, n, &fu));
  std::vector<double> rho(n);
  for (int j = 0; j < n; ++j) rho[j] = (1.0 + mus[j]) / (1.0 - mus[j]);
  // r0 = b - A x0 with A x0 = 2/(1-mu) D x0; a deflated x0 comes with its D x0 combination
  OVL_TRY(copy_convert(c, b, boff, *fq, 0, n));
  if (cfg.defl && cfg.defl->n > 0) {
    std::vector<cd> co;
    OVL_TRY(defl_start(c, cfg.defl, *fq, 0, n, mus, co));
    const int ne = cfg.defl->n;
    // co minimises ||b - D psi co||; this solve is for A = 2 D / (1 - mu), whose
    // minimiser is (1 - mu)/2 co
    for (int i = 0; i < ne; ++i)
      for (int j = 0; j < n; ++j) co[(size_t)i * n + j] *= 0.5 * (1.0 - mus[j]);
    // x = psi co
    OVL_TRY(combine_host(c, cfg.defl->v, 0, ne, co, x, xoff, n, 0));
    // q -= A x0 = 2/(1-mu) ((1+mu)/2 psi co + (1-mu)/2 w co)
    std::vector<cd> cv((size_t)ne * n), cw((size_t)ne * n);
    for (int i = 0; i < ne; ++i)
      for (int j = 0; j < n; ++j) {
        const double f = 2.0 / (1.0 - mus[j]);
        cv[(size_t)i * n + j] = -f * 0.5 * (1.0 + mus[j]) * co[(size_t)i * n + j];
        cw[(size_t)i * n + j] = -f * 0.5 * (1.0 - mus[j]) * co[(size_t)i * n + j];
      }
    OVL_TRY(combine_host(c, cfg.defl->v, 0, ne, cv, *fq, 0, n, 1));
    OVL_TRY(combine_host(c, cfg.defl->w, 0, ne, cw, *fq, 0, n, 1));
  } else {
    launch_zero(x.prec, x.ref(xoff), n, V, c->st);
  }
  std::vector<double> bnorm, delta;
  OVL_TRY(norms_batch(c, b, boff, n, bnorm));
  OVL_TRY(norms_batch(c, *fq, 0, n, delta));
  // normalise q, q~ = q, p = S = 0
  {
    std::vector<cd> a(n), z(n, 0.0);
    for (int j = 0; j < n; ++j) a[j] = delta[j] > 0 ? 1.0 / delta[j] : 0.0;
    OVL_TRY(axpby_batch(c, a, *fq, 0, z, *fq, 0, *fq, 0, n));
    OVL_TRY(copy_convert(c, *fq, 0, *fqt, 0, n));
    launch_zero(PS, fp->ref(), n, V, c->st);
    launch_zero(PS, fS->ref(), n, V, c->st);
  }
  // per-system recurrence state
  struct St : SumrRec {
    bool active = true;
  };
  std::vector<St> S(n);
  res.iters.assign(n, 0);
  res.resid.assign(n, 0.0);
  res.wcalls.assign(n, 0);
  res.sign_calls.assign(n, 0);
  res.stopped.assign(n, 0);
  for (int j = 0; j < n; ++j) {
    S[j].ghat = delta[j];
    S[j].active = delta[j] > cfg.target * bnorm[j] && delta[j] > 0;
    res.resid[j] = delta[j];
  }
  std::vector<double> sc(18 * n);
  std::vector<double> act_d(n);
  std::vector<double> eta(n), dots(4 * n);
  int* d_act = c->dint;
  for (int iter = 0; iter < cfg.maxit; ++iter) {
    int nact = 0;
    double emin = 1e300;
    for (int j = 0; j < n; ++j) {
      if (!S[j].active) {
        eta[j] = 1.0;
        continue;
      }
      ++nact;
      const double r = std::abs(S[j].ghat);
      double e = cfg.relax * cfg.target * bnorm[j] / std::max(r, 1e-300);
      e = std::min(e, cfg.floor);
      if (cfg.eta_cap > 0) e = std::min(e, cfg.eta_cap);
      if (cfg.eta_fixed > 0) e = cfg.eta_fixed;
      if (cfg.eta_dyn) e = *cfg.eta_dyn;
      eta[j] = e;
      emin = std::min(emin, e);
    }
    if (nact == 0) break;
    const int mode = cfg.mode >= 0 ? cfg.mode : choose_mode(c, emin);
    // u = V q = gamma5 eps(K) q, fused with (q~, u), ||u||^2, ||q~||^2
    SignStats ss;
    OVL_TRY(sign_op(c, mode, *fq, 0, *fu, 0, n, eta.data(), 0.0, 1.0, nullptr, 0, fqt, 0, dots.data(), &ss));
    for (int j = 0; j < n; ++j)
      if (S[j].active) {
        res.wcalls[j] += (long long)(2 * ss.iters[j] + 1) * (mode == SIGN64 || mode == SIGN64E ? 2 : 1);
        res.sign_calls[j] += 1;
      }
    if (cfg.hook) OVL_TRY(cfg.hook(c, cfg.hook_data, *fq, *fu, iter));
    std::vector<int> hact(n);
    for (int j = 0; j < n; ++j) {
      double* o = &sc[18 * j];
      for (int k = 0; k < 18; ++k) o[k] = 0.0;
      hact[j] = S[j].active ? 1 : 0;
      if (!S[j].active) continue;
      St& s = S[j];
      cd gam;
      double sig;
      if (!sumr_basis_step(cd(dots[4 * j], dots[4 * j + 1]), dots[4 * j + 2], dots[4 * j + 3], &gam, &sig)) {
        // Krylov space exhausted or a non-finite sign: stop this system here
        s.active = false;
        hact[j] = 0;
        res.stopped[j] = 2;
        continue;
      }
      cd v6[6];
      sumr_rec_step(s, rho[j], gam, sig, v6);
      const cd vals[9] = {v6[0], v6[1], v6[2], v6[3], v6[4], v6[5], gam, 1.0 / sig, sig};
      for (int k = 0; k < 9; ++k) {
        o[2 * k] = vals[k].real();
        o[2 * k + 1] = vals[k].imag();
      }
      if (log_level() >= 3) {
        fprintf(stderr, "  sumr sys %d it %d vals", j, s.it);
        for (int k = 0; k < 9; ++k) fprintf(stderr, " (%.6f,%.6f)", vals[k].real(), vals[k].imag());
        fprintf(stderr, "\n");
      }
      res.iters[j] = s.it;
    }
    const double* dsc;
    OVL_TRY(upload(c, sc.data(), 18 * n, &dsc));
    OVL_CUDA(c, cudaMemcpyAsync(d_act, hact.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
    OVL_TRY(ensure_partials(c, n));
    ProfPair pp;
    prof_begin(c, 4, &pp);
    launch_sumr_update(PS, dsc, d_act, x.ref(xoff), fq->ref(), fqt->ref(), fp->ref(), fS->ref(), fu->ref(), n, V,
                       c->partials, c->st);
    prof_end(c, &pp, (double)nact * V * (double)spinor_site_bytes(PS) * 11.0);
    OVL_TRY(check_launch(c, __func__));
    std::vector<double> qn(2 * n);
    OVL_TRY(reduce_to_host(c, make_shape(V, n).nsb, n, qn.data()));   // also orders the hact upload
    for (int j = 0; j < n; ++j) {
      if (!hact[j]) continue;
      St& s = S[j];
      res.resid[j] = std::abs(s.ghat);
      if (cfg.hist) cfg.hist[j].push_back(std::abs(s.ghat) / bnorm[j]);
      const double qnorm = std::sqrt(std::max(0.0, qn[2 * j]));
      if (log_level() >= 2)
        fprintf(stderr, "  sumr sys %d it %d |r|/|b| %.3e eta %.2e mode %d |q| %.6f gamma %.4f%+.4fi\n", j, s.it,
                std::abs(s.ghat) / bnorm[j], eta[j], mode, qnorm, s.gprev.real(), s.gprev.imag());
      if (std::abs(s.ghat) <= cfg.target * bnorm[j]) {
        s.active = false;
      } else if (std::fabs(qnorm - 1.0) > cfg.qdrift) {
        // the normalisation of q drifts when the sign is inexact (Sec. 2): end this
        // middle solve here; the outer GMRESR step restarts from the true residual
        s.active = false;
        res.stopped[j] = 1;
      }
    }
  }
  return OVL_OK;
}

// ------------------------------------------------------------------ multi-mass relSUMR
// relSUMR for nm masses sharing the Alg. 1 basis of each of ns sources: rho_k + V has the
// Krylov space of V whatever rho_k (Sec. 2: SUMR is adapted to many shifts without
// effort), so q_j, q~_j, gamma_j and sigma_j, and the one sign application per step that
// produces them, serve every mass; only the Givens QR of rho_k + B and the vectors p, S, x
// are per mass. System k ns + j solves (rho_k + V) x = b_j from x = 0 (no deflated start:
// that would give every mass its own residual). The relaxation follows the mass with the
// largest residual, so that every mass gets a sign at least as accurate as it asks for.
ovl_status sumr_multimass(ovl_ctx* c, const SumrCfg& cfg, int ns, int nm, const std::vector<double>& mus_m,
                          const Field& b, int boff, Field& x, int xoff, SumrResult& res) {
  const int PS = cfg.prec;
  const int V = c->V;
  const int n = ns * nm;
  Field *fq, *fqt, *fp, *fS, *fu;
  OVL_TRY(get_field(c, "s_q", PS, ns, &fq));
  OVL_TRY(get_field(c, "s_qt", PS, ns, &fqt));
  OVL_TRY(get_field(c, "s_p", PS, n, &fp));
  OVL_TRY(get_field(c, "s_S", PS, n, &fS));
  OVL_TRY(get_field(c, "s_u", PS, ns, &fu));
  std::vector<double> rho(nm);
  for (int k = 0; k < nm; ++k) rho[k] = (1.0 + mus_m[k]) / (1.0 - mus_m[k]);
  OVL_TRY(copy_convert(c, b, boff, *fq, 0, ns));
  launch_zero(x.prec, x.ref(xoff), n, V, c->st);
  std::vector<double> bnorm;
  OVL_TRY(norms_batch(c, b, boff, ns, bnorm));
  {
    std::vector<cd> a(ns), z(ns, 0.0);
    for (int j = 0; j < ns; ++j) a[j] = bnorm[j] > 0 ? 1.0 / bnorm[j] : 0.0;
    OVL_TRY(axpby_batch(c, a, *fq, 0, z, *fq, 0, *fq, 0, ns));
    OVL_TRY(copy_convert(c, *fq, 0, *fqt, 0, ns));
    launch_zero(PS, fp->ref(), n, V, c->st);
    launch_zero(PS, fS->ref(), n, V, c->st);
  }
  struct St : SumrRec {
    bool active = true;
  };
  std::vector<St> S(n);
  std::vector<char> qact(ns, 0);
  res.iters.assign(n, 0);
  res.resid.assign(n, 0.0);
  res.wcalls.assign(n, 0);
  res.sign_calls.assign(n, 0);
  res.stopped.assign(n, 0);
  for (int k = 0; k < nm; ++k)
    for (int j = 0; j < ns; ++j) {
      St& t = S[k * ns + j];
      t.ghat = bnorm[j];
      t.active = bnorm[j] > 0 && bnorm[j] > cfg.target * bnorm[j];
      res.resid[k * ns + j] = bnorm[j];
      if (t.active) qact[j] = 1;
    }
  std::vector<double> sc(18 * (size_t)n), scq(6 * (size_t)ns);
  std::vector<double> eta(ns), dots(4 * ns);
  std::vector<int> hact(n), hq(ns);
  int* d_act = c->dint;
  int* d_qact = c->dint + 2048;
  for (int iter = 0; iter < cfg.maxit; ++iter) {
    int nq = 0;
    double emin = 1e300;
    for (int j = 0; j < ns; ++j) {
      if (!qact[j]) {
        eta[j] = 1.0;
        continue;
      }
      ++nq;
      double rmax = 0.0;
      for (int k = 0; k < nm; ++k)
        if (S[k * ns + j].active) rmax = std::max(rmax, std::abs(S[k * ns + j].ghat));
      double e = cfg.relax * cfg.target * bnorm[j] / std::max(rmax, 1e-300);
      e = std::min(e, cfg.floor);
      if (cfg.eta_cap > 0) e = std::min(e, cfg.eta_cap);
      if (cfg.eta_fixed > 0) e = cfg.eta_fixed;
      eta[j] = e;
      emin = std::min(emin, e);
    }
    if (nq == 0) break;
    const int mode = cfg.mode >= 0 ? cfg.mode : choose_mode(c, emin);
    SignStats ss;
    OVL_TRY(sign_op(c, mode, *fq, 0, *fu, 0, ns, eta.data(), 0.0, 1.0, nullptr, 0, fqt, 0, dots.data(), &ss));
    // a shared sign application is charged once, split over the masses that use it
    for (int j = 0; j < ns; ++j) {
      int na = 0;
      for (int k = 0; k < nm; ++k) na += S[k * ns + j].active ? 1 : 0;
      if (na == 0) continue;
      const long long cost = (long long)(2 * ss.iters[j] + 1) * (mode == SIGN64 || mode == SIGN64E ? 2 : 1);
      for (int k = 0, seen = 0; k < nm; ++k)
        if (S[k * ns + j].active) {
          res.wcalls[k * ns + j] += cost / na + (seen < cost % na ? 1 : 0);
          res.sign_calls[k * ns + j] += 1;
          ++seen;
        }
    }
    std::fill(sc.begin(), sc.end(), 0.0);
    for (int j = 0; j < ns; ++j) {
      hq[j] = qact[j] ? 1 : 0;
      for (int k = 0; k < nm; ++k) hact[k * ns + j] = qact[j] && S[k * ns + j].active ? 1 : 0;
      if (!qact[j]) continue;
      // the basis step of Alg. 1 with an inexact sign, shared by the masses
      cd gam;
      double sig;
      if (!sumr_basis_step(cd(dots[4 * j], dots[4 * j + 1]), dots[4 * j + 2], dots[4 * j + 3], &gam, &sig)) {
        qact[j] = 0;
        hq[j] = 0;
        for (int k = 0; k < nm; ++k) {
          if (S[k * ns + j].active) res.stopped[k * ns + j] = 2;
          S[k * ns + j].active = false;
          hact[k * ns + j] = 0;
        }
        continue;
      }
      const cd qv[3] = {gam, 1.0 / sig, sig};
      for (int m = 0; m < 3; ++m) {
        scq[6 * j + 2 * m] = qv[m].real();
        scq[6 * j + 2 * m + 1] = qv[m].imag();
      }
      for (int k = 0; k < nm; ++k) {
        St& t = S[k * ns + j];
        if (!t.active) continue;
        cd vals[6];
        sumr_rec_step(t, rho[k], gam, sig, vals);
        double* o = &sc[18 * (size_t)(k * ns + j)];
        for (int m = 0; m < 6; ++m) {
          o[2 * m] = vals[m].real();
          o[2 * m + 1] = vals[m].imag();
        }
        res.iters[k * ns + j] = t.it;
      }
    }
    const double *dsc, *dscq;
    OVL_TRY(upload(c, sc.data(), 18 * n, &dsc));
    OVL_TRY(upload(c, scq.data(), 6 * ns, &dscq));
    OVL_CUDA(c, cudaMemcpyAsync(d_act, hact.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
    OVL_CUDA(c, cudaMemcpyAsync(d_qact, hq.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, c->st));
    OVL_TRY(ensure_partials(c, ns));
    ProfPair pp;
    prof_begin(c, 4, &pp);
    launch_sumr_mm_update(PS, dsc, dscq, d_act, d_qact, x.ref(xoff), fq->ref(), fqt->ref(), fp->ref(), fS->ref(),
                          fu->ref(), ns, nm, V, c->partials, c->st);
    double nact = 0;
    for (int q = 0; q < n; ++q) nact += hact[q];
    prof_end(c, &pp, (double)V * (double)spinor_site_bytes(PS) * (5.0 * nq + 6.0 * nact));
    OVL_TRY(check_launch(c, __func__));
    std::vector<double> qn(2 * ns);
    OVL_TRY(reduce_to_host(c, make_shape(V, ns).nsb, ns, qn.data()));
    for (int j = 0; j < ns; ++j) {
      if (!hq[j]) continue;
      const double qnorm = std::sqrt(std::max(0.0, qn[2 * j]));
      bool any = false;
      for (int k = 0; k < nm; ++k) {
        St& t = S[k * ns + j];
        if (!hact[k * ns + j]) continue;
        res.resid[k * ns + j] = std::abs(t.ghat);
        if (cfg.hist) cfg.hist[k * ns + j].push_back(std::abs(t.ghat) / bnorm[j]);
        if (std::abs(t.ghat) <= cfg.target * bnorm[j]) t.active = false;
        any = any || t.active;
      }
      if (any && std::fabs(qnorm - 1.0) > cfg.qdrift) {
        for (int k = 0; k < nm; ++k)
          if (S[k * ns + j].active) {
            S[k * ns + j].active = false;
            res.stopped[k * ns + j] = 1;
          }
        any = false;
      }
      qact[j] = any ? 1 : 0;
    }
  }
  return OVL_OK;
}

// ------------------------------------------------------------------ relCG (Alg. 4)
// Hhat^-1 x = x + sum_i psi_i (c/sqrt(mu_i) - 1) (psi_i, x), per system mass.
static ovl_status spectral_apply(ovl_ctx* c, ovl_defl* d, const std::vector<double>& mus, Field& x, int xoff, int n) {
  if (!d || d->n == 0) return OVL_OK;
  OVL_TRY(defl_prepare(c, d));
  const int ne = d->n;
  std::vector<cd> G;
  OVL_TRY(gram_host(c, d->v, 0, ne, x, xoff, n, 0, G));
  std::vector<cd> C((size_t)ne * n);
  for (int j = 0; j < n; ++j) {
    std::vector<cd> M;
    dd_matrix(ne, d->VV.data(), d->WW.data(), d->WV.data(), mus[j], M);
    for (int i = 0; i < ne; ++i) {
      const double mui = std::max(M[(size_t)i * ne + i].real() / std::max(d->VV[(size_t)i * ne + i].real(), 1e-300), 1e-300);
      const double f = c->P.c_spec / std::sqrt(mui) - 1.0;
      C[(size_t)i * n + j] = f * G[(size_t)i * n + j];
    }
  }
  return combine_host(c, d->v, 0, ne, C, x, xoff, n, 1);
}

ovl_status cg_batch(ovl_ctx* c, const SumrCfg& cfg, int n, const std::vector<double>& mus, const Field& b, int boff,
                    Field& x, int xoff, SumrResult& res) {
  const int PS = cfg.prec;
  const int V = c->V;
  Field *fr, *fp, *fz, *ft, *fxj;
  OVL_TRY(get_field(c, "c_r", PS, n, &fr));
  OVL_TRY(get_field(c, "c_p", PS, n, &fp));
  OVL_TRY(get_field(c, "c_z", PS, n, &fz));
  OVL_TRY(get_field(c, "c_t", PS, n, &ft));
  OVL_TRY(get_field(c, "c_x", PS, n, &fxj));
  // H x = gamma5 b: r0 = p0 = Hhat^-1 gamma5 b
  OVL_TRY(copy_convert(c, b, boff, *fr, 0, n));
  launch_gamma5(PS, fr->ref(), n, V, c->st);
  OVL_TRY(spectral_apply(c, cfg.defl, mus, *fr, 0, n));
  OVL_TRY(copy_convert(c, *fr, 0, *fp, 0, n));
  launch_zero(PS, fxj->ref(), n, V, c->st);
  std::vector<double> bnorm, rn;
  OVL_TRY(norms_batch(c, b, boff, n, bnorm));
  OVL_TRY(norms_batch(c, *fr, 0, n, rn));
  std::vector<double> rr(n), zeta(n, 0.0);
  std::vector<char> active(n);
  res.iters.assign(n, 0);
  res.resid.assign(n, 0.0);
  res.wcalls.assign(n, 0);
  res.sign_calls.assign(n, 0);
  res.stopped.assign(n, 0);
  for (int j = 0; j < n; ++j) {
    rr[j] = rn[j] * rn[j];
    zeta[j] = rr[j] > 0 ? 1.0 / rr[j] : 0.0;
    active[j] = rn[j] >= cfg.target * bnorm[j] && rn[j] > 0;
    res.resid[j] = rn[j];
  }
  std::vector<double> eta(n);
  std::vector<cd> beta_prev(n, 0.0);
  for (int iter = 0; iter < cfg.maxit; ++iter) {
    int nact = 0;
    double emin = 1e300;
    for (int j = 0; j < n; ++j) {
      double e = cfg.relax * cfg.target * bnorm[j] * std::sqrt(zeta[j]);
      e = std::min(e, cfg.floor);
      if (cfg.eta_cap > 0) e = std::min(e, cfg.eta_cap);
      eta[j] = active[j] ? e : 1.0;
      if (active[j]) {
        ++nact;
        emin = std::min(emin, e);
      }
    }
    if (nact == 0) break;
    const int mode = cfg.mode >= 0 ? cfg.mode : choose_mode(c, emin);
    // z = Hhat^-1 H H Hhat^-1 p
    OVL_TRY(copy_convert(c, *fp, 0, *ft, 0, n));
    OVL_TRY(spectral_apply(c, cfg.defl, mus, *ft, 0, n));
    std::vector<long long> wc(n, 0);
    OVL_TRY(overlap_apply_batch(c, *ft, 0, *fz, 0, n, mus, eta, 1, mode, wc.data()));
    if (cfg.cg_hook) OVL_TRY(cfg.cg_hook(c, cfg.hook_data, *ft, *fz, beta_prev, rn, iter));
    OVL_TRY(overlap_apply_batch(c, *fz, 0, *ft, 0, n, mus, eta, 1, mode, wc.data()));
    OVL_TRY(spectral_apply(c, cfg.defl, mus, *ft, 0, n));
    std::vector<cd> rz;
    OVL_TRY(dots_batch(c, *fr, 0, *ft, 0, n, rz));
    std::vector<cd> al(n, 0.0), one(n, 1.0), mal(n, 0.0);
    for (int j = 0; j < n; ++j) {
      if (!active[j]) continue;
      res.wcalls[j] += wc[j];
      res.sign_calls[j] += 2;
      al[j] = rr[j] / rz[j];
      mal[j] = -al[j];
    }
    OVL_TRY(axpby_batch(c, one, *fr, 0, mal, *ft, 0, *fr, 0, n));   // r -= alpha z
    OVL_TRY(axpby_batch(c, one, *fxj, 0, al, *fp, 0, *fxj, 0, n));  // x += alpha p
    OVL_TRY(norms_batch(c, *fr, 0, n, rn));
    std::vector<cd> beta(n, 0.0);
    for (int j = 0; j < n; ++j) {
      if (!active[j]) {
        beta[j] = 0.0;
        continue;
      }
      const double rrn = rn[j] * rn[j];
      beta[j] = rrn / rr[j];
      rr[j] = rrn;
      zeta[j] += rrn > 0 ? 1.0 / rrn : 0.0;
      res.iters[j] += 1;
      res.resid[j] = rn[j];
      if (rn[j] < cfg.target * bnorm[j]) active[j] = 0;
    }
    std::vector<cd> onea(n, 1.0);
    for (int j = 0; j < n; ++j)
      if (!active[j] && res.iters[j] > 0) {
        // frozen systems: p = r + 0 p keeps them unchanged in value semantics
      }
    OVL_TRY(axpby_batch(c, onea, *fr, 0, beta, *fp, 0, *fp, 0, n));  // p = r + beta p
    beta_prev = beta;
  }
  // x = H Hhat^-1 x_j at the accuracy of the middle solve
  OVL_TRY(spectral_apply(c, cfg.defl, mus, *fxj, 0, n));
  std::vector<double> efin(n, std::min(cfg.floor, cfg.target));
  std::vector<long long> wc(n, 0);
  OVL_TRY(overlap_apply_batch(c, *fxj, 0, x, xoff, n, mus, efin, 1, -1, wc.data()));
  for (int j = 0; j < n; ++j) {
    res.wcalls[j] += wc[j];
    res.sign_calls[j] += 1;
  }
  return OVL_OK;
}

// ------------------------------------------------------------------ GMRESR (Alg. 3)
ovl_status gmresr_batch(ovl_ctx* c, int n, const std::vector<double>& mus, const Field& b, int boff, Field& x,
                        int xoff, double tol, ovl_defl* defl, ovl_solve_info* info, EigHook* eig, int nsrc) {
  auto t0 = std::chrono::steady_clock::now();
  const int V = c->V;
  const int kmax = std::max(1, c->P.gmresr_max);
  const int PS = c->P.mixed ? P32 : P64;
  Field *fr, *fmid_b, *fmid_x, *fu, *fc;
  // the stored directions C_k, U_k get one workspace per outer step, allocated when the
  // step is reached (GMRESR needs 3-4 steps here; reserving gmresr_max of them for a
  // large batch would take tens of GB)
  std::vector<Field*> fC, fU;
  OVL_TRY(get_field(c, "g_r", P64, n, &fr));
  OVL_TRY(get_field(c, "g_u", P64, n, &fu));
  OVL_TRY(get_field(c, "g_c", P64, n, &fc));
  OVL_TRY(get_field(c, "m_b", PS, n, &fmid_b));
  OVL_TRY(get_field(c, "m_x", PS, n, &fmid_x));
  // x = 0, r = b
  launch_zero(P64, x.ref(xoff), n, V, c->st);
  OVL_TRY(copy_convert(c, b, boff, *fr, 0, n));
  std::vector<double> bn, rn;
  OVL_TRY(norms_batch(c, b, boff, n, bn));
  rn = bn;
  const double eta_t = c->P.eta_precond > 0 ? c->P.eta_precond : std::cbrt(tol);
  // The outer loop stops at half the requested tolerance: the recursive residual and the
  // true one differ by the sign errors allowed in c = A u (below), and the reported true
  // residual is itself measured with a sign of finite accuracy, so stopping at tol itself
  // would leave the true residual at tol to within those errors, on either side.
  const double tstop = 0.5 * tol;
  std::vector<char> active(n);
  std::vector<int> outer(n, 0), inner(n, 0), signs(n, 0);
  std::vector<long long> wcalls(n, 0);
  for (int j = 0; j < n; ++j) active[j] = rn[j] > tstop * bn[j];
  for (int k = 0; k < kmax; ++k) {
    int nact = 0;
    for (int j = 0; j < n; ++j) nact += active[j];
    if (nact == 0) break;
    // middle solve A u = r to relative accuracy eta~ (all systems in the batch advance;
    // converged ones are solved for their tiny residual, which costs iterations only
    // while others still run)
    OVL_TRY(copy_convert(c, *fr, 0, *fmid_b, 0, n));
    SumrCfg cfg;
    cfg.prec = PS;
    cfg.target = (eig && eig->active) ? eig->target : eta_t;
    cfg.relax = c->P.relax_factor;
    cfg.floor = c->P.eta_floor;
    cfg.maxit = c->P.inner_max;
    cfg.defl = defl;
    cfg.mode = -1;
    cfg.qdrift = 0.1;
    cfg.eta_cap = (eig && eig->active) ? eig->eta_cap : 0.0;
    if (eig && eig->active) {
      cfg.hook = eig->hook;
      cfg.cg_hook = eig->cg_hook;
      cfg.hook_data = eig->data;
    }
    SumrResult sr;
    // first outer step of a batch that holds every mass of its sources (system q =
    // mass * nsrc + source, x = 0 so r = b): the masses share one SUMR basis per source
    bool mm = k == 0 && nsrc > 0 && n % nsrc == 0 && n / nsrc > 1 && !defl && !(eig && eig->active) &&
              c->P.solver != OVL_SOLVER_CG;
    std::vector<double> mus_m;
    if (mm) {
      for (int m = 0; m < n / nsrc; ++m) {
        mus_m.push_back(mus[m * nsrc]);
        for (int j = 1; j < nsrc; ++j) mm = mm && mus[m * nsrc + j] == mus[m * nsrc];
      }
    }
    if (c->P.solver == OVL_SOLVER_CG) OVL_TRY(cg_batch(c, cfg, n, mus, *fmid_b, 0, *fmid_x, 0, sr));
    else if (mm) OVL_TRY(sumr_multimass(c, cfg, nsrc, n / nsrc, mus_m, *fmid_b, 0, *fmid_x, 0, sr));
    else OVL_TRY(sumr_batch(c, cfg, n, mus, *fmid_b, 0, *fmid_x, 0, sr));
    OVL_TRY(copy_convert(c, *fmid_x, 0, *fu, 0, n));
    if (c->P.solver != OVL_SOLVER_CG) {
      // SUMR solved (rho + V) u = r, i.e. D u = (1-mu)/2 r: rescale u by 2/(1-mu)
      std::vector<cd> a(n), z(n, 0.0);
      for (int j = 0; j < n; ++j) a[j] = 2.0 / (1.0 - mus[j]);
      OVL_TRY(axpby_batch(c, a, *fu, 0, z, *fu, 0, *fu, 0, n));
    }
    for (int j = 0; j < n; ++j)
      if (active[j]) {
        inner[j] += sr.iters[j];
        wcalls[j] += sr.wcalls[j];
        signs[j] += sr.sign_calls[j];
      }
    // c = A u with ||A u - c|| < eps ||b|| ||u|| / ||r||
    std::vector<double> eta(n);
    double emin = 1e300;
    for (int j = 0; j < n; ++j) {
      // Alg. 3 bounds ||A u - c|| relative to ||u||; through the update r -= alpha c that
      // error reaches r amplified by up to ||u|| / ||A u|| <= 1/mu (D^dag D >= mu^2), so
      // the factor mu/2 keeps the final true residual within tol
      eta[j] = active[j] ? std::min(c->P.eta_floor, 0.5 * mus[j] * tstop * bn[j] / std::max(rn[j], 1e-300))
                         : c->P.eta_floor;
      emin = std::min(emin, eta[j]);
    }
    std::vector<long long> wc(n, 0);
    OVL_TRY(overlap_apply_batch(c, *fu, 0, *fc, 0, n, mus, eta, 0, -1, wc.data()));
    for (int j = 0; j < n; ++j)
      if (active[j]) {
        wcalls[j] += wc[j];
        signs[j] += 1;
      }
    // orthogonalise against the stored C (same combination on u)
    for (int i = 0; i < k; ++i) {
      std::vector<cd> beta;
      OVL_TRY(dots_batch(c, *fC[i], 0, *fc, 0, n, beta));
      std::vector<cd> one(n, 1.0), mb(n);
      for (int j = 0; j < n; ++j) mb[j] = -beta[j];
      OVL_TRY(axpby_batch(c, one, *fc, 0, mb, *fC[i], 0, *fc, 0, n));
      OVL_TRY(axpby_batch(c, one, *fu, 0, mb, *fU[i], 0, *fu, 0, n));
    }
    std::vector<double> nu;
    OVL_TRY(norms_batch(c, *fc, 0, n, nu));
    {
      std::vector<cd> a(n), z(n, 0.0);
      for (int j = 0; j < n; ++j) a[j] = nu[j] > 0 ? 1.0 / nu[j] : 0.0;
      Field *ck, *uk;
      OVL_TRY(get_field(c, "g_C" + std::to_string(k), P64, n, &ck));
      OVL_TRY(get_field(c, "g_U" + std::to_string(k), P64, n, &uk));
      fC.push_back(ck);
      fU.push_back(uk);
      OVL_TRY(axpby_batch(c, a, *fc, 0, z, *fc, 0, *fC[k], 0, n));
      OVL_TRY(axpby_batch(c, a, *fu, 0, z, *fu, 0, *fU[k], 0, n));
    }
    std::vector<cd> alpha;
    OVL_TRY(dots_batch(c, *fC[k], 0, *fr, 0, n, alpha));
    {
      std::vector<cd> one(n, 1.0), al(n), mal(n);
      for (int j = 0; j < n; ++j) {
        al[j] = active[j] ? alpha[j] : 0.0;
        mal[j] = -al[j];
      }
      OVL_TRY(axpby_batch(c, one, x, xoff, al, *fU[k], 0, x, xoff, n));
      OVL_TRY(axpby_batch(c, one, *fr, 0, mal, *fC[k], 0, *fr, 0, n));
    }
    OVL_TRY(norms_batch(c, *fr, 0, n, rn));
    if (log_level() >= 1)
      for (int j = 0; j < n; ++j)
        fprintf(stderr, "gmresr step %d sys %d |r|/|b| %.3e middle iters %d stopped %d |u| nu %.3e alpha %.3e%+.3ei\n",
                k, j, rn[j] / bn[j], sr.iters[j], sr.stopped[j], nu[j], alpha[j].real(), alpha[j].imag());
    for (int j = 0; j < n; ++j)
      if (active[j]) {
        outer[j] += 1;
        if (rn[j] <= tstop * bn[j]) active[j] = 0;
      }
    if (eig && eig->after_outer) OVL_TRY(eig->after_outer(c, eig->data, k));
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) {
    for (int j = 0; j < n; ++j) {
      ovl_solve_info& I = info[j];
      I.converged = rn[j] <= tol * bn[j];
      I.outer_iters = outer[j];
      I.inner_iters = inner[j];
      I.sign_calls = signs[j];
      I.wilson_calls = wcalls[j];
      I.true_residual = bn[j] > 0 ? rn[j] / bn[j] : 0.0;
      I.seconds = secs;
    }
  }
  for (int j = 0; j < n; ++j)
    if (!std::isfinite(rn[j])) return set_err(c, OVL_EBREAKDOWN, "GMRESR residual is not finite");
  for (int j = 0; j < n; ++j)
    if (rn[j] > tol * bn[j]) return set_err(c, OVL_ENOCONV, "GMRESR did not reach the tolerance");
  return OVL_OK;
}

}  // namespace ovl
