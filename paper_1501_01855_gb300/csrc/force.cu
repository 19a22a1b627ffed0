// Gauge-link gradient of S = phi^dag (D^dag D)^-1 phi through the Zolotarev
// rational with its coefficients held fixed (the paper has no force; this is the
// derivative of the operator of Secs. 1 and 3).
//
// With H = gamma5 D = (1+mu)/2 gamma5 + (1-mu)/2 eps(K), D^dag D = H^2, chi = H^-2 phi,
// psi = H chi, R_i = (K^2 + sigma_i)^-1, a_i = R_i chi, b_i = R_i K psi:
//   dS = -(1-mu) sum_i omega_i Re[ psi^dag dK a_i - b_i^dag dK (K a_i) - (K b_i)^dag dK a_i ].
// For one link U_mu(s), Re[x^dag dK y] = -kappa Re sum_ab conj(dU_ab) (conj(F_ab) + G_ba),
//   F_ab = sum_spin conj(P+ x(s))_{a} (P- y(s+mu))_{b},  G_ab = sum_spin conj(P- x(s+mu))_{a} (P+ y(s))_{b},
// where P-+ are the half-spinor projections of (1 -+ gamma_mu) (gamma5 (1 -+ gamma_mu) sandwiched
// between x and y reduces to them). The result G_link is defined by dS = 2 Re sum conj(G) dU.
//
// Every shifted solution comes from a multi-shift CG that keeps the individual x_i: all
// poles at once when their fields fit in HBM, else in groups of poles solved one after
// the other (recomputed, not stored; params.force_pole_group).
// The outer-product kernel runs over all poles in one pass with an FP64
// accumulator per link (compute in FP64, or FP32 with the mixed setting).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "context.h"
#include "solver.h"

namespace ovl {

template <int MU, int S, typename T>
__device__ __forceinline__ void halfproj(const cpx<T> p[12], cpx<T> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cpx<T> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if constexpr (MU == 0) {
      h[c] = S > 0 ? p0 + timesI(p3) : p0 - timesI(p3);
      h[3 + c] = S > 0 ? p1 + timesI(p2) : p1 - timesI(p2);
    } else if constexpr (MU == 1) {
      h[c] = S > 0 ? p0 - p3 : p0 + p3;
      h[3 + c] = S > 0 ? p1 + p2 : p1 - p2;
    } else if constexpr (MU == 2) {
      h[c] = S > 0 ? p0 + timesI(p2) : p0 - timesI(p2);
      h[3 + c] = S > 0 ? p1 - timesI(p3) : p1 + timesI(p3);
    } else {
      h[c] = S > 0 ? p0 + p2 : p0 - p2;
      h[3 + c] = S > 0 ? p1 + p3 : p1 - p3;
    }
  }
}

// acc_ab += w * (conj(F_ab) + G_ba) for the link (s, MU)
template <int MU, typename T>
__device__ __forceinline__ void link_term(const cpx<T> xs[12], const cpx<T> ys[12], const cpx<T> xf[12],
                                          const cpx<T> yf[12], double w, cpx<double> acc[9]) {
  cpx<T> hx[6], hy[6], gx[6], gy[6];
  halfproj<MU, +1>(xs, hx);   // P+ x(s)
  halfproj<MU, -1>(yf, hy);   // P- y(s+mu)
  halfproj<MU, -1>(xf, gx);   // P- x(s+mu)
  halfproj<MU, +1>(ys, gy);   // P+ y(s)
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // F_ab = sum_sp conj(hx[sp,a]) hy[sp,b];  G_ba = sum_sp conj(gx[sp,b]) gy[sp,a]
      const cpx<T> F = cmulc(hx[a], hy[b]) + cmulc(hx[3 + a], hy[3 + b]);
      const cpx<T> G = cmulc(gx[b], gy[a]) + cmulc(gx[3 + b], gy[3 + a]);
      acc[3 * a + b].r += w * ((double)F.r + (double)G.r);
      acc[3 * a + b].i += w * (-(double)F.i + (double)G.i);
    }
}

template <int MU, typename T>
__device__ __forceinline__ void force_dir(const Geom& g, int s, int sf, bool wrapt, SpinorRef psi, SpinorRef a,
                                          SpinorRef Ka, SpinorRef b, SpinorRef Kb, int np, const double* coef,
                                          double kappa, double* G) {
  cpx<double> acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = cmk(0.0, 0.0);
  cpx<T> x0[12], x1[12], y0[12], y1[12];
  const T sgn = (MU == 3 && g.bc_t && wrapt) ? T(-1) : T(1);
  cpx<T> ps[12], pf[12];
  load_spinor_as<P64, T>(psi, 0, s, ps);
  load_spinor_as<P64, T>(psi, 0, sf, pf);
#pragma unroll
  for (int k = 0; k < 12; ++k) pf[k] = sgn * pf[k];
  for (int i = 0; i < np; ++i) {
    const double w = -0.5 * kappa * coef[i];
    // psi^dag dK a_i
    load_spinor_as<P64, T>(a, i, s, y0);
    load_spinor_as<P64, T>(a, i, sf, y1);
#pragma unroll
    for (int k = 0; k < 12; ++k) y1[k] = sgn * y1[k];
    link_term<MU, T>(ps, y0, pf, y1, w, acc);
    // -(K b_i)^dag dK a_i
    load_spinor_as<P64, T>(Kb, i, s, x0);
    load_spinor_as<P64, T>(Kb, i, sf, x1);
#pragma unroll
    for (int k = 0; k < 12; ++k) x1[k] = sgn * x1[k];
    link_term<MU, T>(x0, y0, x1, y1, -w, acc);
    // -b_i^dag dK (K a_i)
    load_spinor_as<P64, T>(b, i, s, x0);
    load_spinor_as<P64, T>(b, i, sf, x1);
    load_spinor_as<P64, T>(Ka, i, s, y0);
    load_spinor_as<P64, T>(Ka, i, sf, y1);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      x1[k] = sgn * x1[k];
      y1[k] = sgn * y1[k];
    }
    link_term<MU, T>(x0, y0, x1, y1, -w, acc);
  }
  double* out = G + (((size_t)s * 4 + MU) * 9) * 2;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    out[2 * k] += acc[k].r;
    out[2 * k + 1] += acc[k].i;
  }
}

template <typename T>
__global__ void __launch_bounds__(128) force_kernel(Geom g, double kappa, SpinorRef psi, SpinorRef a, SpinorRef Ka,
                                                    SpinorRef b, SpinorRef Kb, int np, const double* coef, double* G) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  int t = s;
  x[0] = t % g.L[0]; t /= g.L[0];
  x[1] = t % g.L[1]; t /= g.L[1];
  x[2] = t % g.L[2]; x[3] = t / g.L[2];
  const int st[4] = {1, g.L[0], g.L[0] * g.L[1], g.L[0] * g.L[1] * g.L[2]};
  int sf[4];
  bool wr[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    wr[mu] = x[mu] == g.L[mu] - 1;
    sf[mu] = wr[mu] ? s - (g.L[mu] - 1) * st[mu] : s + st[mu];
  }
  force_dir<0, T>(g, s, sf[0], wr[0], psi, a, Ka, b, Kb, np, coef, kappa, G);
  force_dir<1, T>(g, s, sf[1], wr[1], psi, a, Ka, b, Kb, np, coef, kappa, G);
  force_dir<2, T>(g, s, sf[2], wr[2], psi, a, Ka, b, Kb, np, coef, kappa, G);
  force_dir<3, T>(g, s, sf[3], wr[3], psi, a, Ka, b, Kb, np, coef, kappa, G);
}

void launch_force(int fp32, const Geom& g, double kappa, SpinorRef psi, SpinorRef a, SpinorRef Ka, SpinorRef b,
                  SpinorRef Kb, int npoles, const double* coef, double* G, cudaStream_t st) {
  const int nb = (g.V + 127) / 128;
  if (fp32) force_kernel<float><<<nb, 128, 0, st>>>(g, kappa, psi, a, Ka, b, Kb, npoles, coef, G);
  else force_kernel<double><<<nb, 128, 0, st>>>(g, kappa, psi, a, Ka, b, Kb, npoles, coef, G);
}

// The shifted solutions (K^2 + sigma_i) x_i = v of one group of np poles (device data dpol,
// base shift sigma0 = the group's smallest) to relative residual tol, FP64.
static ovl_status shifted_solutions(ovl_ctx* c, const Field& v, Field& xs, double tol, Poles* dpol, int np,
                                    double sigma0) {
  const int V = c->V;
  Field *r, *pb;
  OVL_TRY(get_field(c, "f_r", P64, 1, &r));
  OVL_TRY(get_field(c, "f_p", P64, np, &pb));
  Field* t;
  OVL_TRY(get_field(c, "f_t", P64, 1, &t));
  OVL_TRY(ensure_partials(c, 1));
  OVL_TRY(ensure_ms(c, 1));
  launch_zero(P64, xs.ref(), np, V, c->st);
  Field* y;
  OVL_TRY(get_field(c, "f_y", P64, 1, &y));
  launch_ms_init(P64, P64, P64, v.ref(), r->ref(), pb->ref(), y->ref(), np, 1, V, c->partials, c->st);
  // with unit weights the stopping rule bounds sum_i |zeta_i| ||r|| (plus the poles
  // already stopped) by eta ||v||: eta = tol makes every shifted system accurate to tol
  c->hpin[0] = tol;
  OVL_CUDA(c, cudaMemcpyAsync(c->dscal, c->hpin, sizeof(double), cudaMemcpyHostToDevice, c->st));
  const Shape sh = make_shape(V, 1);
  launch_ms_scalar0(c->ms, c->partials, sh.nsb, 1, dpol, c->dscal, c->P.mscg_max, c->st);
  const LinkRef L = links_of(c, P64);
  int* hd = reinterpret_cast<int*>(c->hpin + 8192);
  int total = 0;
  while (true) {
    for (int k = 0; k < 8; ++k) {
      launch_wilson_K(P64, P64, P64, c->g, c->kappa, L, pb->ref(), t->ref(), 1, c->partials, c->ms, c->st);
      launch_ms_scalar1(c->ms, c->partials, sh.nsb, 1, dpol, c->st);
      launch_wilson_mscg_r(P64, P64, P64, P64, c->g, c->kappa, L, t->ref(), pb->ref(), r->ref(), 1, sigma0,
                           c->partials, c->ms, c->st);
      launch_ms_scalar2(c->ms, c->partials, sh.nsb, 1, dpol, c->st);
      launch_ms_update_x(r->ref(), pb->ref(), xs.ref(), np, 1, V, c->ms, c->st);
    }
    total += 8;
    OVL_TRY(check_launch(c, __func__));
    OVL_CUDA(c, cudaMemcpyAsync(hd, &c->ms[0].done, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    OVL_CUDA(c, cudaStreamSynchronize(c->st));
    if (hd[0] || total > c->P.mscg_max + 16) break;
  }
  c->wcalls[P64] += 2 * total;
  OVL_CUDA(c, cudaMemcpyAsync(hd, &c->ms[0].status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaMemcpyAsync(hd + 1, &c->ms[0].iter, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  if (hd[0] != 0) {
    char m[200];
    snprintf(m, sizeof(m), "shifted solves of the gradient: multi-shift CG %s after %d iterations (tolerance %.3e)",
             hd[0] == 2 ? "broke down" : "reached the iteration limit mscg_max", hd[1], tol);
    return set_err(c, hd[0] == 2 ? OVL_EBREAKDOWN : OVL_ENOCONV, m);
  }
  return OVL_OK;
}

ovl_status force_compute(ovl_ctx* c, double mu, const Field& phi, double tol, double* dSdU, double* S) {
  const int np = c->npoles, V = c->V;
  // chi = D^-1 gamma5 D^-1 gamma5 phi   ((D^dag)^-1 = gamma5 D^-1 gamma5)
  Field *g1, *x1, *chi, *psi, *Kpsi;
  OVL_TRY(get_field(c, "f_g1", P64, 1, &g1));
  OVL_TRY(get_field(c, "f_x1", P64, 1, &x1));
  OVL_TRY(get_field(c, "f_chi", P64, 1, &chi));
  OVL_TRY(get_field(c, "f_psi", P64, 1, &psi));
  OVL_TRY(get_field(c, "f_Kpsi", P64, 1, &Kpsi));
  std::vector<double> mus(1, mu);
  ovl_params keep = c->P;
  c->P.verify = 0;
  // every sign below evaluates the rational itself to tol, not just to within Delta
  struct ExactScope {
    ovl_ctx* c;
    ~ExactScope() { c->exact_rational = false; }
  } scope{c};
  c->exact_rational = true;
  const double stol = tol;
  OVL_TRY(copy_convert(c, phi, 0, *g1, 0, 1));
  launch_gamma5(P64, g1->ref(), 1, V, c->st);
  ovl_status s1 = gmresr_batch(c, 1, mus, *g1, 0, *x1, 0, stol, nullptr, nullptr, nullptr);
  if (s1 != OVL_OK) {
    c->P = keep;
    return s1;
  }
  launch_gamma5(P64, x1->ref(), 1, V, c->st);
  s1 = gmresr_batch(c, 1, mus, *x1, 0, *chi, 0, stol, nullptr, nullptr, nullptr);
  c->P = keep;
  if (s1 != OVL_OK) return s1;
  if (S) {
    std::vector<cd> d;
    OVL_TRY(dots_batch(c, phi, 0, *chi, 0, 1, d));
    *S = d[0].real();
  }
  // psi = H chi, K psi
  std::vector<double> eta(1, tol * 0.1);
  OVL_TRY(overlap_apply_batch(c, *chi, 0, *psi, 0, 1, mus, eta, 1, SIGN64, nullptr));
  OVL_TRY(wilson_apply_field(c, P64, *psi, 0, *Kpsi, 0, 1));
  // The shifted solutions of chi and K psi (unit pole weights for the stopping rule), in
  // groups of g poles: all at once when their 5 g fields (A, K A, B, K B and the
  // multi-shift directions) fit in half the free device memory, else as many as fit; each
  // group is solved afresh (recomputed rather than stored) and its terms added to G.
  int g = c->P.force_pole_group;
  if (g <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      fr = 0;
    }
    const double per = 5.0 * V * 192.0;
    g = fr == 0 ? np : (int)std::max(1.0, std::min((double)np, 0.5 * (double)fr / per));
  }
  g = std::min(g, np);
  std::vector<double> coef(np);
  for (int i = 0; i < np; ++i) coef[i] = -(1.0 - mu) * c->omega[i];
  const double* dcoef;
  OVL_TRY(upload(c, coef.data(), np, &dcoef));
  const size_t nG = (size_t)V * 4 * 9 * 2;
  OVL_TRY(ensure_work(c, nG));
  OVL_CUDA(c, cudaMemsetAsync(c->dwork, 0, nG * sizeof(double), c->st));
  Field *A, *KA, *B, *KB;
  OVL_TRY(get_field(c, "f_A", P64, g, &A));
  OVL_TRY(get_field(c, "f_KA", P64, g, &KA));
  OVL_TRY(get_field(c, "f_B", P64, g, &B));
  OVL_TRY(get_field(c, "f_KB", P64, g, &KB));
  Poles* dfp;
  OVL_CUDA(c, cudaMalloc((void**)&dfp, sizeof(Poles)));
  ovl_status st = OVL_OK;
  for (int i0 = 0; i0 < np && st == OVL_OK; i0 += g) {
    const int gn = std::min(g, np - i0);
    Poles fp;
    memset(&fp, 0, sizeof(fp));
    fp.n = gn;
    fp.sigma0 = c->sigma[i0];
    for (int i = 0; i < gn; ++i) {
      fp.ds[i] = c->sigma[i0 + i] - c->sigma[i0];
      fp.omega[i] = 1.0;
      fp.gbound[i] = 1.0;
    }
    // the previous group's kernels read dfp: update it in stream order
    cudaStreamSynchronize(c->st);
    cudaMemcpy(dfp, &fp, sizeof(Poles), cudaMemcpyHostToDevice);
    st = shifted_solutions(c, *chi, *A, tol * 0.1, dfp, gn, fp.sigma0);
    if (st == OVL_OK) st = shifted_solutions(c, *Kpsi, *B, tol * 0.1, dfp, gn, fp.sigma0);
    if (st == OVL_OK) st = wilson_apply_field(c, P64, *A, 0, *KA, 0, gn);
    if (st == OVL_OK) st = wilson_apply_field(c, P64, *B, 0, *KB, 0, gn);
    if (st != OVL_OK) break;
    ProfPair pp;
    prof_begin(c, 7, &pp);
    launch_force(c->P.mixed ? 1 : 0, c->g, c->kappa, psi->ref(), A->ref(), KA->ref(), B->ref(), KB->ref(), gn,
                 dcoef + i0, c->dwork, c->st);
    prof_end(c, &pp, (double)V * (192.0 * (1 + 4.0 * gn) + nG / V * 8.0));
    st = check_launch(c, __func__);
  }
  cudaStreamSynchronize(c->st);
  cudaFree(dfp);
  if (st != OVL_OK) return st;
  OVL_CUDA(c, cudaMemcpyAsync(dSdU, c->dwork, nG * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  return OVL_OK;
}

}  // namespace ovl
