// The C ABI of liboverlap (declared in include/overlap.h).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>

#include "context.h"
#include "eig.h"
#include "hostmath.h"
#include "solver.h"

using namespace ovl;

namespace ovl {
ovl_status force_compute(ovl_ctx* c, double mu, const Field& phi, double tol, double* dSdU, double* S);
}

static const char* kVersion = "liboverlap 0.1 (sm_103a)";

extern "C" const char* ovl_version(void) { return kVersion; }

extern "C" ovl_status ovl_params_default(ovl_params* p) {
  if (!p) return OVL_EINVAL;
  memset(p, 0, sizeof(*p));
  p->solver = OVL_SOLVER_SUMR;
  p->mixed = 1;
  p->half_storage = 0;
  p->emulate_fp64 = 1;
  p->eta_floor = 1e-2;
  p->sp_switch = 1e-6;
  p->half_switch = 2e-3;
  p->eta_precond = 0.0;
  p->relax_factor = 1.0;
  p->gmresr_max = 30;
  p->inner_max = 2000;
  p->mscg_max = 5000;
  p->delta_split = 0.01;
  p->c_spec = std::sqrt(3.0) / 2.0;
  p->bc_t = 0;
  p->a_override = 0.0;
  p->b_override = 0.0;
  p->batch_max = 36;
  p->wilson_variant = -1;
  p->use_graphs = 1;
  p->verify = 1;
  p->sign_method = 0;
  p->basis_gb = 96.0;
  p->multimass = 1;
  p->force_pole_group = 0;
  p->lanczos_cap = 0;
  p->gram_method = 0;
  p->stream = nullptr;
  return OVL_OK;
}

extern "C" const char* overlap_last_error(const ovl_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" ovl_status ovl_trim(ovl_ctx* c) {
  if (!c) return OVL_EINVAL;
  trim_workspaces(c);
  return OVL_OK;
}

// ---------------------------------------------------------------- create
static void convert_links(const double* links, const int L[4], int bc_t, std::vector<double>& l64,
                          std::vector<float>& l32, std::vector<__half>& l16, std::vector<float>& l64e) {
  const int V = L[0] * L[1] * L[2] * L[3];
  // canonical [site][mu][row][col] complex -> [mu][chunk][V] keeping rows 0, 1.
  // The double-float copy holds, for each site x, the matrix of each of the eight hops
  // in slot n = 2 mu + b: b = 0 U_mu(x), b = 1 U_mu(x - mu)^dag, all 9 entries
  // ([n][chunk][V]), with the antiperiodic-t sign of the hops that cross the boundary
  // folded in.
  l64.assign((size_t)4 * 6 * V * 2, 0.0);
  l32.assign((size_t)4 * 3 * V * 4, 0.f);
  l16.assign((size_t)4 * 3 * V * 4, __float2half(0.f));
  l64e.assign((size_t)8 * 9 * V * 4, 0.f);
  auto put_df = [&](int n, int e, int s, double re, double im) {
    const float rh = (float)re, ih = (float)im;
    float* d = &l64e[(((size_t)n * 9 + e) * V + s) * 4];
    d[0] = rh;
    d[1] = (float)(re - (double)rh);
    d[2] = ih;
    d[3] = (float)(im - (double)ih);
  };
  const int str[4] = {1, L[0], L[0] * L[1], L[0] * L[1] * L[2]};
  for (int s = 0; s < V; ++s) {
    int x[4], r = s;
    for (int d = 0; d < 4; ++d) {
      x[d] = r % L[d];
      r /= L[d];
    }
    for (int mu = 0; mu < 4; ++mu) {
      const double* u = links + ((size_t)s * 4 + mu) * 18;   // 9 complex
      const int sb = x[mu] == 0 ? s + (L[mu] - 1) * str[mu] : s - str[mu];
      const double* ub = links + ((size_t)sb * 4 + mu) * 18;
      const double sf = (mu == 3 && bc_t && x[3] == L[3] - 1) ? -1.0 : 1.0;
      const double sbk = (mu == 3 && bc_t && x[3] == 0) ? -1.0 : 1.0;
      for (int e = 0; e < 9; ++e) {
        put_df(2 * mu, e, s, sf * u[2 * e], sf * u[2 * e + 1]);
        const int t = 3 * (e % 3) + e / 3;   // (U^dag)_{ab} = conj(U_{ba})
        put_df(2 * mu + 1, e, s, sbk * ub[2 * t], -sbk * ub[2 * t + 1]);
      }
      for (int e = 0; e < 6; ++e) {
        const double re = u[2 * e], im = u[2 * e + 1];
        l64[(((size_t)mu * 6 + e) * V + s) * 2 + 0] = re;
        l64[(((size_t)mu * 6 + e) * V + s) * 2 + 1] = im;
        const int ch = e / 2, w = e % 2;
        l32[(((size_t)mu * 3 + ch) * V + s) * 4 + 2 * w + 0] = (float)re;
        l32[(((size_t)mu * 3 + ch) * V + s) * 4 + 2 * w + 1] = (float)im;
        l16[(((size_t)mu * 3 + ch) * V + s) * 4 + 2 * w + 0] = __float2half_rn((float)re);
        l16[(((size_t)mu * 3 + ch) * V + s) * 4 + 2 * w + 1] = __float2half_rn((float)im);
      }
    }
  }
}

// Create-time autotuner: the Wilson-kernel launch shapes (thread per site, direction split,
// 4D tiles when the lattice divides into them, and for double-float the lane-pair form)
// timed for every storage precision on this lattice (random input), once with one system
// and once with a batch (min(12, batch_max) systems; 4 in double-float), and the fastest
// kept for each (another shape must beat the thread-per-site one by 5%).
static ovl_status autotune_wilson(ovl_ctx* c) {
  const int forced = c->P.wilson_variant;
  std::vector<double> h((size_t)24 * c->V);
  unsigned long long st = 777;
  for (auto& x : h) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    x = ((double)(st >> 11) / 9007199254740992.0) - 0.5;
  }
  cudaEvent_t e0, e1;
  OVL_CUDA(c, cudaEventCreate(&e0));
  OVL_CUDA(c, cudaEventCreate(&e1));
  for (int p = 0; p < 4; ++p) {
    if (forced >= 0 && forced <= 3) {
      c->wvar[p] = (forced == 2 && !wilson_tiles_fit(c->g)) || (forced == 3 && p != P64E) ? 0 : forced;
      c->wvar_multi[p] = c->wvar[p];
      continue;
    }
    const int nmulti = p == P64E ? std::min(4, c->P.batch_max) : std::min(12, c->P.batch_max);
    Field *fi, *fo;
    OVL_TRY(get_field(c, "at_in", p, std::max(1, nmulti), &fi));
    OVL_TRY(get_field(c, "at_out", p, std::max(1, nmulti), &fo));
    for (int j = 0; j < std::max(1, nmulti); ++j) OVL_TRY(import_spinors(c, h.data(), OVL_C128, 0, 1, *fi, j));
    const int nv = p == P64E ? 4 : wilson_tiles_fit(c->g) ? 3 : 2;
    for (int bucket = 0; bucket < 2; ++bucket) {
      const int ns = bucket == 0 ? 1 : nmulti;
      float* wt = bucket == 0 ? c->wtime[p] : c->wtime_multi[p];
      if (bucket == 1 && ns < 4) {
        c->wvar_multi[p] = c->wvar[p];
        break;
      }
      for (int v = 0; v < nv; ++v) {
        if (v == 2 && !wilson_tiles_fit(c->g)) continue;
        LinkRef L = links_of(c, p);
        L.variant = L.variant_multi = v;
        const int reps = p == P64 ? 3 : bucket == 0 ? 8 : 4;
        for (int w = 0; w < 2; ++w)
          launch_wilson_K(p, p, p, c->g, c->kappa, L, fi->ref(), fo->ref(), ns, nullptr, nullptr, c->st);
        OVL_CUDA(c, cudaEventRecord(e0, c->st));
        for (int w = 0; w < reps; ++w)
          launch_wilson_K(p, p, p, c->g, c->kappa, L, fi->ref(), fo->ref(), ns, nullptr, nullptr, c->st);
        OVL_CUDA(c, cudaEventRecord(e1, c->st));
        OVL_CUDA(c, cudaEventSynchronize(e1));
        OVL_TRY(check_launch(c, __func__));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        wt[v] = ms / reps;
      }
      // another shape must beat the thread-per-site one by 5%: closer timings are within
      // run-to-run noise, and the choice should not flip between runs
      int best = 0;
      for (int v = 1; v < nv; ++v)
        if (wt[v] > 0.f && wt[v] < 0.95f * wt[0] && wt[v] < wt[best]) best = v;
      (bucket == 0 ? c->wvar[p] : c->wvar_multi[p]) = best;
    }
    free_field(c->ws["at_in"]);
    free_field(c->ws["at_out"]);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return OVL_OK;
}

// Extreme eigenvalues of K^2 by FP64 Lanczos (no reorthogonalisation; only the
// ends of the spectrum are used).
ovl_status ovl::lanczos_bounds(ovl_ctx* c, int steps, double* lmin, double* lmax, const Field* proj, int nproj) {
  Field *v0, *v1, *w, *t;
  OVL_TRY(get_field(c, "lz_v0", P64, 1, &v0));
  OVL_TRY(get_field(c, "lz_v1", P64, 1, &v1));
  OVL_TRY(get_field(c, "lz_w", P64, 1, &w));
  OVL_TRY(get_field(c, "lz_t", P64, 1, &t));
  std::vector<double> h((size_t)24 * c->V);
  unsigned long long st = 0x9E3779B97F4A7C15ull;
  for (auto& x : h) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    x = ((double)(st >> 11) / 9007199254740992.0) - 0.5;
  }
  OVL_TRY(import_spinors(c, h.data(), OVL_C128, 0, 1, *v1, 0));
  // v <- v - Psi (Psi^dag v): the Krylov space of K^2 on the complement of proj
  auto project = [&](Field& f) -> ovl_status {
    if (!proj || nproj <= 0) return OVL_OK;
    std::vector<cd> G;
    OVL_TRY(gram_host(c, *proj, 0, nproj, f, 0, 1, 0, G));
    for (auto& g : G) g = -g;
    return combine_host(c, *proj, 0, nproj, G, f, 0, 1, 1);
  };
  OVL_TRY(project(*v1));
  std::vector<double> nrm;
  OVL_TRY(norms_batch(c, *v1, 0, 1, nrm));
  std::vector<cd> a1(1, 1.0 / nrm[0]), z1(1, 0.0), one(1, 1.0);
  OVL_TRY(axpby_batch(c, a1, *v1, 0, z1, *v1, 0, *v1, 0, 1));
  launch_zero(P64, v0->ref(), 1, c->V, c->st);
  std::vector<double> al, be;
  double beta = 0.0;
  for (int j = 0; j < steps; ++j) {
    OVL_TRY(wilson_apply_field(c, P64, *v1, 0, *t, 0, 1));
    OVL_TRY(wilson_apply_field(c, P64, *t, 0, *w, 0, 1));
    OVL_TRY(project(*w));
    std::vector<cd> d;
    OVL_TRY(dots_batch(c, *v1, 0, *w, 0, 1, d));
    const double alpha = d[0].real();
    al.push_back(alpha);
    std::vector<cd> ma(1, -alpha), mb(1, -beta);
    OVL_TRY(axpby_batch(c, one, *w, 0, ma, *v1, 0, *w, 0, 1));
    OVL_TRY(axpby_batch(c, one, *w, 0, mb, *v0, 0, *w, 0, 1));
    OVL_TRY(norms_batch(c, *w, 0, 1, nrm));
    beta = nrm[0];
    if (beta < 1e-14) break;
    be.push_back(beta);
    std::swap(c->ws["lz_v0"], c->ws["lz_v1"]);
    v0 = &c->ws["lz_v0"];
    v1 = &c->ws["lz_v1"];
    std::vector<cd> ib(1, 1.0 / beta);
    OVL_TRY(axpby_batch(c, ib, *w, 0, z1, *w, 0, *v1, 0, 1));
    // the three-term recurrence would amplify what is left of the projected directions
    // (their coefficients follow a recurrence of their own): project every new vector
    OVL_TRY(project(*v1));
  }
  const int n = (int)al.size();
  be.resize(std::max(0, n - 1));
  tridiag_extremes(n, al.data(), be.data(), lmin, lmax);
  return OVL_OK;
}

extern "C" void overlap_destroy(ovl_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  for (auto& kv : c->ws) free_field(kv.second);
  free_field(c->kd);
  if (c->lz_pool) cudaFree(c->lz_pool);
  for (int p = 0; p < 4; ++p)
    if (c->link[p]) cudaFree(c->link[p]);
  if (c->partials) cudaFree(c->partials);
  if (c->dred) cudaFree(c->dred);
  if (c->dscal) cudaFree(c->dscal);
  if (c->dint) cudaFree(c->dint);
  if (c->ms) cudaFree(c->ms);
  if (c->lz) cudaFree(c->lz);
  if (c->lz_hist) cudaFree(c->lz_hist);
  if (c->lz_Y) cudaFree(c->lz_Y);
  if (c->lz_coefW) cudaFree(c->lz_coefW);
  if (c->lz_ctr) cudaFree(c->lz_ctr);
  if (c->dpoles) cudaFree(c->dpoles);
  if (c->dwork) cudaFree(c->dwork);
  if (c->hpin) cudaFreeHost(c->hpin);
  if (c->hstage) cudaFreeHost(c->hstage);
  if (c->stage_ev) cudaEventDestroy(c->stage_ev);
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  for (auto& q : c->prof.pending) {
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  for (auto e : c->prof.pool) cudaEventDestroy(e);
  delete c;
}

static ovl_status create_impl(ovl_ctx* c, const int dims[4], const double* links, double m0, double mu, int n_poles,
                              double eps_sign, const ovl_params* params) {
  if (params) c->P = *params;
  else ovl_params_default(&c->P);
  for (int d = 0; d < 4; ++d) {
    if (dims[d] < 2 || (dims[d] & 1)) return set_err(c, OVL_EINVAL, "lattice extents must be even and >= 2");
    c->g.L[d] = dims[d];
  }
  const long long Vll = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  if (Vll > (1LL << 28)) return set_err(c, OVL_EINVAL, "lattice too large");
  c->V = (int)Vll;
  c->g.V = c->V;
  c->g.bc_t = c->P.bc_t ? 1 : 0;
  // multiply-shift constants for site -> coordinate division (see common.cuh)
  for (int d = 0; d < 3; ++d) {
    int l = 0;
    while ((1 << l) < dims[d]) ++l;
    const int k = 31 + l;
    c->g.dk[d] = k;
    c->g.dm[d] = (((unsigned long long)1 << k) + (unsigned long long)dims[d] - 1) / (unsigned long long)dims[d];
  }
  if (!(m0 > 0 && m0 < 4)) return set_err(c, OVL_EINVAL, "m0 must lie in (0, 4)");
  if (!(mu >= 0 && mu < 1)) return set_err(c, OVL_EINVAL, "mu must lie in [0, 1)");
  if (n_poles < 1 || n_poles > NPMAX) return set_err(c, OVL_EINVAL, "n_poles must lie in 1..64");
  if (c->P.sign_method < 0 || c->P.sign_method > 2) return set_err(c, OVL_EINVAL, "sign_method must be 0, 1 or 2");
  if (!(c->P.basis_gb > 0)) c->P.basis_gb = 96.0;
  if (c->P.lanczos_cap != 0 && (c->P.lanczos_cap < 4 || c->P.lanczos_cap > 1024))
    return set_err(c, OVL_EINVAL, "lanczos_cap must be 0 or lie in 4..1024");
  if (c->P.gram_method != 0 && c->P.gram_method != 1) return set_err(c, OVL_EINVAL, "gram_method must be 0 or 1");
  if (c->P.batch_max < 1) c->P.batch_max = 1;
  if (c->P.batch_max > 256) c->P.batch_max = 256;
  c->m0 = m0;
  c->kappa = 1.0 / (8.0 - 2.0 * m0);
  c->mu = mu;
  c->eps_sign = eps_sign;
  c->st = (cudaStream_t)c->P.stream;
  OVL_CUDA(c, cudaGetDevice(&c->device));
  OVL_CUDA(c, cudaMallocHost((void**)&c->hpin, sizeof(double) * 64 * 4096));
  OVL_CUDA(c, cudaMalloc((void**)&c->dscal, sizeof(double) * 64 * 4096));
  OVL_CUDA(c, cudaMalloc((void**)&c->dred, sizeof(double) * NVRED * 4096));
  OVL_CUDA(c, cudaMalloc((void**)&c->dint, sizeof(int) * 4096));
  OVL_CUDA(c, cudaMalloc((void**)&c->dpoles, sizeof(Poles)));
  OVL_CUDA(c, cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming));
  OVL_CUDA(c, cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
  // gauge field in the three storage formats
  {
    std::vector<double> l64;
    std::vector<float> l32;
    std::vector<__half> l16;
    std::vector<float> l64e;
    convert_links(links, c->g.L, c->g.bc_t, l64, l32, l16, l64e);
    OVL_CUDA(c, cudaMalloc(&c->link[P64E], l64e.size() * sizeof(float)));
    OVL_CUDA(c, cudaMemcpy(c->link[P64E], l64e.data(), l64e.size() * sizeof(float), cudaMemcpyHostToDevice));
    OVL_CUDA(c, cudaMalloc(&c->link[P64], l64.size() * sizeof(double)));
    OVL_CUDA(c, cudaMalloc(&c->link[P32], l32.size() * sizeof(float)));
    OVL_CUDA(c, cudaMalloc(&c->link[P16], l16.size() * sizeof(__half)));
    OVL_CUDA(c, cudaMemcpy(c->link[P64], l64.data(), l64.size() * sizeof(double), cudaMemcpyHostToDevice));
    OVL_CUDA(c, cudaMemcpy(c->link[P32], l32.data(), l32.size() * sizeof(float), cudaMemcpyHostToDevice));
    OVL_CUDA(c, cudaMemcpy(c->link[P16], l16.data(), l16.size() * sizeof(__half), cudaMemcpyHostToDevice));
  }
  OVL_TRY(autotune_wilson(c));
  // spectral bounds of |K|
  double a = c->P.a_override, b = c->P.b_override;
  if (!(a > 0) || !(b > 0)) {
    double lmin, lmax;
    OVL_TRY(lanczos_bounds(c, 300, &lmin, &lmax));
    if (!(a > 0)) a = 0.95 * std::sqrt(std::max(lmin, 1e-30));
    if (!(b > 0)) b = 1.05 * std::sqrt(lmax);
  }
  if (!(b > a)) return set_err(c, OVL_EINVAL, "spectral bounds need 0 < a < b");
  OVL_TRY(set_poles(c, n_poles, a, b));
  c->za0 = a;
  c->npoles0 = n_poles;
  return OVL_OK;
}

ovl_status ovl::set_poles(ovl_ctx* c, int n_poles, double a, double b) {
  std::vector<double> om(n_poles), sg(n_poles);
  double delta = 0.0;
  if (zolotarev_coeffs(n_poles, a, b, om.data(), sg.data(), &delta) != 0)
    return set_err(c, OVL_EINVAL, "Zolotarev coefficients failed");
  if (delta > c->eps_sign) {
    char m[200];
    snprintf(m, sizeof(m), "Zolotarev Delta %.3e with %d poles on [%.4g, %.4g] exceeds eps_sign %.3e", delta,
             n_poles, a, b, c->eps_sign);
    return set_err(c, OVL_EAPPROX, m);
  }
  c->npoles = n_poles;
  c->za = a;
  c->zb = b;
  c->omega = om;
  c->sigma = sg;
  c->delta = delta;
  Poles& P = c->hpoles;
  memset(&P, 0, sizeof(P));
  P.n = n_poles;
  P.sigma0 = c->sigma[0];
  for (int i = 0; i < n_poles; ++i) {
    P.ds[i] = c->sigma[i] - c->sigma[0];
    P.omega[i] = c->omega[i];
    P.gbound[i] = pole_gbound(c->sigma[i], a, b);
  }
  if (c->st) cudaStreamSynchronize(c->st);
  OVL_CUDA(c, cudaMemcpy(c->dpoles, &P, sizeof(Poles), cudaMemcpyHostToDevice));
  // step counts seen so far belong to the old rational
  memset(c->lz_kmax, 0, sizeof(c->lz_kmax));
  return OVL_OK;
}

extern "C" ovl_status overlap_create(ovl_ctx** out, const int dims[4], const double* links, double m0, double mu,
                                     int n_poles, double eps_sign, const ovl_params* params) {
  if (!out || !dims || !links) return OVL_EINVAL;
  *out = nullptr;
  ovl_ctx* c = new (std::nothrow) ovl_ctx();
  if (!c) return OVL_ENOMEM;
  ovl_status s = create_impl(c, dims, links, m0, mu, n_poles, eps_sign, params);
  if (s != OVL_OK) {
    // keep the message readable through a static buffer after destroying c
    static thread_local char msg[512];
    snprintf(msg, sizeof(msg), "%s", c->err.c_str());
    fprintf(stderr, "liboverlap: overlap_create failed: %s\n", msg);
    overlap_destroy(c);
    return s;
  }
  *out = c;
  return OVL_OK;
}

extern "C" ovl_status ovl_zolotarev_coeffs(int n, double a, double b, double* omega, double* sigma, double* delta) {
  if (n < 1 || n > NPMAX || !omega || !sigma || !delta || !(a > 0) || !(b > a)) return OVL_EINVAL;
  return zolotarev_coeffs(n, a, b, omega, sigma, delta) == 0 ? OVL_OK : OVL_EINVAL;
}

// The host numerics the solvers run between launches, on caller copies (the helpers
// work in place); complex matrices are row-major interleaved (re, im) doubles, which is
// the layout of std::complex<double>.
static const int HOST_NMAX = 4096;

extern "C" ovl_status ovl_host_eigh(int n, const double* a, double* w, double* z) {
  if (n < 1 || n > HOST_NMAX || !a || !w || !z) return OVL_EINVAL;
  std::vector<cd> A((size_t)n * n);
  memcpy(A.data(), a, sizeof(cd) * (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (!std::isfinite(A[(size_t)i * n + j].real()) || !std::isfinite(A[(size_t)i * n + j].imag())) return OVL_EINVAL;
  eigh_herm(n, A.data(), w, reinterpret_cast<cd*>(z));
  return OVL_OK;
}

extern "C" ovl_status ovl_host_cholesky(int n, const double* a, double* l) {
  if (n < 1 || n > HOST_NMAX || !a || !l) return OVL_EINVAL;
  std::vector<cd> L((size_t)n * n);
  memcpy(L.data(), a, sizeof(cd) * (size_t)n * n);
  if (cholesky_lower(n, L.data()) != 0) return OVL_EBREAKDOWN;
  memcpy(l, L.data(), sizeof(cd) * (size_t)n * n);
  return OVL_OK;
}

extern "C" ovl_status ovl_host_lower_inverse(int n, const double* l, double* li) {
  if (n < 1 || n > HOST_NMAX || !l || !li) return OVL_EINVAL;
  const cd* L = reinterpret_cast<const cd*>(l);
  for (int i = 0; i < n; ++i)
    if (std::abs(L[(size_t)i * n + i]) == 0.0) return OVL_EBREAKDOWN;
  std::vector<cd> Li((size_t)n * n);
  lower_inverse(n, L, Li.data());
  memcpy(li, Li.data(), sizeof(cd) * (size_t)n * n);
  return OVL_OK;
}

extern "C" ovl_status ovl_host_lu_solve(int n, const double* a, const double* b, int nb, double* x) {
  if (n < 1 || n > HOST_NMAX || nb < 1 || nb > HOST_NMAX || !a || !b || !x) return OVL_EINVAL;
  std::vector<cd> A((size_t)n * n), B((size_t)n * nb);
  memcpy(A.data(), a, sizeof(cd) * (size_t)n * n);
  memcpy(B.data(), b, sizeof(cd) * (size_t)n * nb);
  if (lu_solve(n, A.data(), B.data(), nb) != 0) return OVL_EBREAKDOWN;
  memcpy(x, B.data(), sizeof(cd) * (size_t)n * nb);
  return OVL_OK;
}

extern "C" ovl_status ovl_host_tridiag_extremes(int n, const double* d, const double* e, double* lmin,
                                                double* lmax) {
  if (n < 1 || !d || (n > 1 && !e) || !lmin || !lmax) return OVL_EINVAL;
  tridiag_extremes(n, d, e, lmin, lmax);
  return OVL_OK;
}

extern "C" ovl_status ovl_host_sumr_step(double rho, const double* dots, double* state, double* coef) {
  if (!dots || !state || !coef || !(rho > 1.0) || !std::isfinite(rho)) return OVL_EINVAL;
  for (int i = 0; i < 11; ++i)
    if (!std::isfinite(state[i])) return OVL_EINVAL;
  SumrRec r;
  r.gprev = cd(state[0], state[1]);
  r.sprev = cd(state[2], state[3]);
  r.cprev = state[4];
  r.sigprev = state[5];
  r.zeta = cd(state[6], state[7]);
  r.ghat = cd(state[8], state[9]);
  r.it = (int)state[10];
  cd gam;
  double sig;
  if (!sumr_basis_step(cd(dots[0], dots[1]), dots[2], dots[3], &gam, &sig)) return OVL_EBREAKDOWN;
  cd v6[6];
  sumr_rec_step(r, rho, gam, sig, v6);
  const cd vals[9] = {v6[0], v6[1], v6[2], v6[3], v6[4], v6[5], gam, 1.0 / sig, sig};
  for (int k = 0; k < 9; ++k) {
    coef[2 * k] = vals[k].real();
    coef[2 * k + 1] = vals[k].imag();
  }
  const double st[11] = {r.gprev.real(), r.gprev.imag(), r.sprev.real(), r.sprev.imag(), r.cprev, r.sigprev,
                         r.zeta.real(), r.zeta.imag(), r.ghat.real(), r.ghat.imag(), (double)r.it};
  memcpy(state, st, sizeof(st));
  return OVL_OK;
}

extern "C" ovl_status ovl_host_defl_start(int n, const double* VV, const double* WW, const double* WV,
                                          const double* G5VV, const double* G5VW, int nsys, const double* VB,
                                          const double* WB, const double* mus, int per_vector, double* coefs) {
  if (n < 1 || n > 1024 || nsys < 1 || nsys > 4096 || !VV || !WW || !WV || !G5VV || !G5VW || !VB || !WB || !mus ||
      !coefs)
    return OVL_EINVAL;
  for (int j = 0; j < nsys; ++j)
    if (!(mus[j] > 0 && mus[j] < 1)) return OVL_EINVAL;
  const size_t nn = (size_t)2 * n * n, nb = (size_t)2 * n * nsys;
  for (const double* p : {VV, WW, WV, G5VV, G5VW})
    for (size_t i = 0; i < nn; ++i)
      if (!std::isfinite(p[i])) return OVL_EINVAL;
  for (const double* p : {VB, WB})
    for (size_t i = 0; i < nb; ++i)
      if (!std::isfinite(p[i])) return OVL_EINVAL;
  auto C = [](const double* p) { return reinterpret_cast<const cd*>(p); };
  return defl_start_host(n, C(VV), C(WW), C(WV), C(G5VV), C(G5VW), nsys, C(VB), C(WB), mus, per_vector != 0,
                         reinterpret_cast<cd*>(coefs));
}

extern "C" ovl_status ovl_host_ritz(int k, const double* E, const double* MVD, const double* G5, double mu,
                                    double delta, int keep, int restart, double* ritz, double* C, double* res,
                                    int* kept) {
  if (k < 1 || k > 1024 || keep < 1 || keep > k || !E || !MVD || !G5 || !ritz || !C || !res || !kept)
    return OVL_EINVAL;
  if (!(mu > 0 && mu < 1) || !(delta >= 0)) return OVL_EINVAL;
  const size_t kk2 = (size_t)2 * k * k;
  for (const double* p : {E, MVD, G5})
    for (size_t i = 0; i < kk2; ++i)
      if (!std::isfinite(p[i])) return OVL_EINVAL;
  RitzHost rh;
  ritz_host(k, reinterpret_cast<const cd*>(E), reinterpret_cast<const cd*>(MVD), reinterpret_cast<const cd*>(G5), mu,
            delta, keep, restart != 0, &rh);
  *kept = rh.keep;
  memcpy(ritz, rh.lam.data(), sizeof(double) * rh.keep);
  memcpy(res, rh.res.data(), sizeof(double) * rh.keep);
  memcpy(C, rh.C.data(), sizeof(cd) * (size_t)k * rh.keep);
  return OVL_OK;
}

extern "C" ovl_status overlap_zolotarev(const ovl_ctx* c, double* omega, double* sigma, double* delta, double* a,
                                        double* b) {
  if (!c) return OVL_EINVAL;
  if (omega) memcpy(omega, c->omega.data(), sizeof(double) * c->npoles);
  if (sigma) memcpy(sigma, c->sigma.data(), sizeof(double) * c->npoles);
  if (delta) *delta = c->delta;
  if (a) *a = c->za;
  if (b) *b = c->zb;
  return OVL_OK;
}

static ovl_status check_io(ovl_ctx* c, const void* in, const void* out, int n, int dtype) {
  if (!c) return OVL_EINVAL;
  if (!in || !out) return set_err(c, OVL_EINVAL, "null spinor pointer");
  if (n < 1 || n > 4096) return set_err(c, OVL_EINVAL, "n must lie in 1..4096");
  if (dtype != OVL_C128 && dtype != OVL_C64) return set_err(c, OVL_EINVAL, "dtype must be OVL_C128 or OVL_C64");
  return OVL_OK;
}

extern "C" ovl_status ovl_wilson_apply(ovl_ctx* c, const void* in, void* out, int n, int dtype, int on_device,
                                       int prec) {
  OVL_TRY(check_io(c, in, out, n, dtype));
  if (prec < P64 || prec > P64E) return set_err(c, OVL_EINVAL, "prec must be OVL_PREC_F64, F32, F16 or F64E");
  Field *fi, *fo;
  OVL_TRY(get_field(c, "api_wi", prec, n, &fi));
  OVL_TRY(get_field(c, "api_wo", prec, n, &fo));
  OVL_TRY(import_spinors(c, in, dtype, on_device, n, *fi, 0));
  OVL_TRY(wilson_apply_field(c, prec, *fi, 0, *fo, 0, n));
  OVL_TRY(export_spinors(c, out, dtype, on_device, n, *fo, 0));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  return OVL_OK;
}

extern "C" ovl_status ovl_sign_apply(ovl_ctx* c, const void* in, void* out, int n, int dtype, int on_device,
                                     double eta, int prec) {
  OVL_TRY(check_io(c, in, out, n, dtype));
  Field *fi, *fo;
  OVL_TRY(get_field(c, "api_in", P64, n, &fi));
  OVL_TRY(get_field(c, "api_out", P64, n, &fo));
  OVL_TRY(import_spinors(c, in, dtype, on_device, n, *fi, 0));
  const double e = eta > 0 ? eta : c->eps_sign;
  const int mode = prec == OVL_PREC_AUTO ? choose_mode(c, e) : prec;
  if (mode < SIGN64 || mode > SIGN64E) return set_err(c, OVL_EINVAL, "bad prec");
  std::vector<double> etas(n, e);
  OVL_TRY(sign_op(c, mode, *fi, 0, *fo, 0, n, etas.data(), 0.0, 1.0, nullptr, 1, nullptr, 0, nullptr, nullptr));
  OVL_TRY(export_spinors(c, out, dtype, on_device, n, *fo, 0));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  return OVL_OK;
}

extern "C" ovl_status overlap_apply(ovl_ctx* c, double mu, const void* in, void* out, int n, int dtype, int on_device,
                                    double eta, int prec, int hermitian) {
  OVL_TRY(check_io(c, in, out, n, dtype));
  if (!(mu >= 0 && mu < 1)) return set_err(c, OVL_EINVAL, "mu must lie in [0, 1)");
  Field *fi, *fo;
  OVL_TRY(get_field(c, "api_in", P64, n, &fi));
  OVL_TRY(get_field(c, "api_out", P64, n, &fo));
  OVL_TRY(import_spinors(c, in, dtype, on_device, n, *fi, 0));
  const double e = eta > 0 ? eta : c->eps_sign;
  const int mode = prec == OVL_PREC_AUTO ? choose_mode(c, e) : prec;
  if (mode < SIGN64 || mode > SIGN64E) return set_err(c, OVL_EINVAL, "bad prec");
  std::vector<double> mus(n, mu), etas(n, e);
  OVL_TRY(overlap_apply_batch(c, *fi, 0, *fo, 0, n, mus, etas, hermitian ? 1 : 0, mode, nullptr));
  OVL_TRY(export_spinors(c, out, dtype, on_device, n, *fo, 0));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  return OVL_OK;
}

extern "C" ovl_status overlap_sumr(ovl_ctx* c, double mu, const void* b, void* x, int n, int dtype, int on_device,
                                   double tol, double eta_fixed, int maxit, double* hist, int* iters) {
  OVL_TRY(check_io(c, b, x, n, dtype));
  if (!(mu > 0 && mu < 1)) return set_err(c, OVL_EINVAL, "mu must lie in (0, 1)");
  if (maxit < 1 || !(tol > 0)) return set_err(c, OVL_EINVAL, "need maxit >= 1 and tol > 0");
  const int PS = c->P.mixed ? P32 : P64;
  Field *fb, *fx, *fo;
  OVL_TRY(get_field(c, "api_in", P64, n, &fb));
  OVL_TRY(get_field(c, "sm_b", PS, n, &fx));
  OVL_TRY(get_field(c, "sm_x", PS, n, &fo));
  OVL_TRY(import_spinors(c, b, dtype, on_device, n, *fb, 0));
  OVL_TRY(copy_convert(c, *fb, 0, *fx, 0, n));
  SumrCfg cfg;
  cfg.prec = PS;
  cfg.target = tol;
  cfg.relax = c->P.relax_factor;
  cfg.floor = c->P.eta_floor;
  cfg.maxit = maxit;
  cfg.eta_fixed = eta_fixed;
  std::vector<std::vector<double>> h(n);
  cfg.hist = h.data();
  std::vector<double> mus(n, mu);
  SumrResult sr;
  OVL_TRY(sumr_batch(c, cfg, n, mus, *fx, 0, *fo, 0, sr));
  // (rho + V) x' = b  ->  D x = b with x = 2 x' / (1 - mu)
  Field* fr;
  OVL_TRY(get_field(c, "api_out", P64, n, &fr));
  OVL_TRY(copy_convert(c, *fo, 0, *fr, 0, n));
  std::vector<cd> a(n, 2.0 / (1.0 - mu)), z(n, 0.0);
  OVL_TRY(axpby_batch(c, a, *fr, 0, z, *fr, 0, *fr, 0, n));
  OVL_TRY(export_spinors(c, x, dtype, on_device, n, *fr, 0));
  for (int j = 0; j < n; ++j) {
    if (iters) iters[j] = sr.iters[j];
    if (hist)
      for (int k = 0; k < maxit; ++k) hist[(size_t)j * maxit + k] = k < (int)h[j].size() ? h[j][k] : 0.0;
  }
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  return OVL_OK;
}

// true residual ||b - D x|| / ||b|| with an FP64 sign at eps_sign
// ||b - D x|| / ||b|| with a sign accurate enough to resolve tol: its error enters as
// (1 - mu)/2 eta ||x||, and ||x|| can reach ||b|| / mu.
static ovl_status true_residuals(ovl_ctx* c, const Field& b, int boff, const Field& x, int xoff, int n,
                                 const std::vector<double>& mus, double tol, std::vector<double>& out) {
  Field* t;
  OVL_TRY(get_field(c, "tr_t", P64, n, &t));
  std::vector<double> etas(n);
  for (int j = 0; j < n; ++j) etas[j] = std::min(c->eps_sign, 0.1 * tol * mus[j]);
  OVL_TRY(overlap_apply_batch(c, x, xoff, *t, 0, n, mus, etas, 0, c->P.emulate_fp64 ? SIGN64E : SIGN64, nullptr));
  std::vector<cd> one(n, 1.0), mone(n, -1.0);
  OVL_TRY(axpby_batch(c, one, b, boff, mone, *t, 0, *t, 0, n));
  std::vector<double> rn, bn;
  OVL_TRY(norms_batch(c, *t, 0, n, rn));
  OVL_TRY(norms_batch(c, b, boff, n, bn));
  out.resize(n);
  for (int j = 0; j < n; ++j) {
    out[j] = bn[j] > 0 ? rn[j] / bn[j] : 0.0;
    if (!std::isfinite(out[j])) {
      char m[160];
      snprintf(m, sizeof(m), "the true residual of system %d is not finite (the verification sign failed)", j);
      return set_err(c, OVL_EBREAKDOWN, m);
    }
  }
  return OVL_OK;
}

extern "C" ovl_status overlap_solve(ovl_ctx* c, int nrhs, const double* mus, int nmass, const void* rhs, void* x,
                                    int dtype, int on_device, double tol, ovl_defl* defl, ovl_solve_info* info) {
  OVL_TRY(check_io(c, rhs, x, nrhs, dtype));
  if (nmass < 1 || nmass > 64) return set_err(c, OVL_EINVAL, "nmass must lie in 1..64");
  if (!(tol > 0)) return set_err(c, OVL_EINVAL, "tol must be positive");
  std::vector<double> mv(nmass);
  for (int k = 0; k < nmass; ++k) {
    mv[k] = mus ? mus[k] : c->mu;
    if (!(mv[k] > 0 && mv[k] < 1)) return set_err(c, OVL_EINVAL, "every mass must lie in (0, 1)");
  }
  if (defl && defl->ctx != c) return set_err(c, OVL_EINVAL, "deflation space belongs to another context");
  Field* fb;
  OVL_TRY(get_field(c, "api_b", P64, nrhs, &fb));
  OVL_TRY(import_spinors(c, rhs, dtype, on_device, nrhs, *fb, 0));
  const int nsys = nrhs * nmass;
  const int bm = std::max(1, c->P.batch_max);
  const size_t esz = (dtype == OVL_C128 ? 16 : 8) * 12 * (size_t)c->V;
  ovl_status worst = OVL_OK;
  // undeflated relSUMR with several masses: batches of whole sources (every mass), so that
  // the first middle solve shares one SUMR basis per source
  if (c->P.multimass && nmass > 1 && !defl && c->P.solver != OVL_SOLVER_CG && nmass <= bm) {
    const int nsb = std::max(1, bm / nmass);
    for (int j0 = 0; j0 < nrhs; j0 += nsb) {
      const int nj = std::min(nsb, nrhs - j0), n = nj * nmass;
      Field *bb, *bx;
      OVL_TRY(get_field(c, "bat_b", P64, n, &bb));
      OVL_TRY(get_field(c, "bat_x", P64, n, &bx));
      std::vector<double> bmus(n);
      for (int k = 0; k < nmass; ++k)
        for (int jl = 0; jl < nj; ++jl) {
          bmus[k * nj + jl] = mv[k];
          OVL_TRY(copy_convert(c, *fb, j0 + jl, *bb, k * nj + jl, 1));
        }
      std::vector<ovl_solve_info> binfo(n);
      ovl_status st = gmresr_batch(c, n, bmus, *bb, 0, *bx, 0, tol, nullptr, binfo.data(), nullptr, nj);
      if (st != OVL_OK && st != OVL_ENOCONV) return st;
      if (st == OVL_ENOCONV) worst = st;
      if (c->P.verify) {
        std::vector<double> tr;
        OVL_TRY(true_residuals(c, *bb, 0, *bx, 0, n, bmus, tol, tr));
        for (int q = 0; q < n; ++q) {
          binfo[q].true_residual = tr[q];
          binfo[q].converged = tr[q] <= tol * 1.0000001 ? 1 : 0;
        }
      }
      for (int k = 0; k < nmass; ++k) {
        char* dst = (char*)x + esz * ((size_t)k * nrhs + j0);
        OVL_TRY(export_spinors(c, dst, dtype, on_device, nj, *bx, k * nj));
        if (info)
          for (int jl = 0; jl < nj; ++jl) info[(size_t)k * nrhs + j0 + jl] = binfo[k * nj + jl];
      }
    }
    OVL_CUDA(c, cudaStreamSynchronize(c->st));
    if (info)
      for (int s = 0; s < nsys; ++s) info[s].wilson_f64 = info[s].wilson_f32 = info[s].wilson_f16 = 0;
    return worst;
  }
  for (int s0 = 0; s0 < nsys; s0 += bm) {
    const int n = std::min(bm, nsys - s0);
    Field *bb, *bx;
    OVL_TRY(get_field(c, "bat_b", P64, n, &bb));
    OVL_TRY(get_field(c, "bat_x", P64, n, &bx));
    std::vector<double> bmus(n);
    for (int q = 0; q < n; ++q) {
      const int s = s0 + q;
      const int k = s / nrhs, j = s % nrhs;
      bmus[q] = mv[k];
      OVL_TRY(copy_convert(c, *fb, j, *bb, q, 1));
    }
    ovl_status st = gmresr_batch(c, n, bmus, *bb, 0, *bx, 0, tol, defl, info ? info + s0 : nullptr, nullptr);
    if (st != OVL_OK && st != OVL_ENOCONV) return st;
    if (st == OVL_ENOCONV) worst = st;
    if (c->P.verify) {
      std::vector<double> tr;
      OVL_TRY(true_residuals(c, *bb, 0, *bx, 0, n, bmus, tol, tr));
      if (info)
        for (int q = 0; q < n; ++q) {
          info[s0 + q].true_residual = tr[q];
          info[s0 + q].converged = tr[q] <= tol * 1.0000001 ? 1 : 0;
          info[s0 + q].wilson_calls += 0;
        }
    }
    char* dst = (char*)x + esz * s0;
    OVL_TRY(export_spinors(c, dst, dtype, on_device, n, *bx, 0));
  }
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  if (info) {
    for (int s = 0; s < nsys; ++s) {
      info[s].wilson_f64 = info[s].wilson_f32 = info[s].wilson_f16 = 0;
    }
  }
  return worst;
}

// ---------------------------------------------------------------- eigSUMR
static ovl_status defl_alloc(ovl_ctx* c, ovl_defl* d, int prec, int cap) {
  d->ctx = c;
  d->cap = cap;
  auto alloc = [&](Field& f) -> ovl_status {
    f.prec = prec;
    f.V = c->V;
    f.n = cap;
    if (cudaMalloc(&f.data, (size_t)spinor_site_bytes(prec) * c->V * cap) != cudaSuccess) {
      cudaGetLastError();
      f.data = nullptr;
      return set_err(c, OVL_ENOMEM, "cudaMalloc failed for the deflation space");
    }
    return OVL_OK;
  };
  OVL_TRY(alloc(d->v));
  OVL_TRY(alloc(d->w));
  return OVL_OK;
}

extern "C" void ovl_defl_destroy(ovl_defl* d) {
  if (!d) return;
  if (d->ctx && d->ctx->st) cudaStreamSynchronize(d->ctx->st);
  free_field(d->v);
  free_field(d->w);
  delete d;
}

// Store the first nk vectors of V as the space d, recompute w = gamma5 eps(K) psi
// accurately (Sec. 5.1: v^D is recalculated after the eigenvector calculation, before
// the space is used), and take the Ritz values of D^dag D + 2 mu delta H and the residuals
// ||gamma5 D psi - psi (psi, gamma5 D psi)|| from the recomputed w.
static ovl_status defl_store(ovl_ctx* c, ovl_defl* d, const Field* V, int nk, double mu) {
  if (d->cap < nk) return set_err(c, OVL_EINVAL, "internal: deflation capacity");
  OVL_TRY(copy_convert(c, *V, 0, d->v, 0, nk));
  std::vector<double> etas(nk, std::max(c->eps_sign, 1e-8));
  const int mode = choose_mode(c, etas[0]);
  OVL_TRY(sign_op(c, mode, d->v, 0, d->w, 0, nk, etas.data(), 0.0, 1.0, nullptr, 0, nullptr, 0, nullptr, nullptr));
  d->n = nk;
  d->mu = mu;
  d->prepared = false;
  OVL_TRY(defl_prepare(c, d));
  d->ritz.assign(nk, 0.0);
  d->res.assign(nk, 0.0);
  const double a = 0.5 * (1.0 - mu), b = 0.5 * (1.0 + mu);
  for (int i = 0; i < nk; ++i) {
    const size_t ii = (size_t)i * nk + i;
    const double vv = d->VV[ii].real();
    const cd wv = d->WV[ii];
    const double dd = a * a * d->WW[ii].real() + 2.0 * a * b * wv.real() + b * b * vv;   // ||D psi||^2
    const cd th = b * d->G5VV[ii] + a * d->G5VW[ii];                                    // (psi, g5 D psi)
    d->ritz[i] = (dd + 2.0 * mu * c->P.delta_split * th.real()) / vv;
    d->res[i] = std::sqrt(std::max(0.0, dd / vv - std::norm(th) / (vv * vv)));
  }
  return OVL_OK;
}

static ovl_status eig_after_outer(ovl_ctx* c, void* data, int outer) {
  (void)c;
  (void)data;
  (void)outer;
  return OVL_OK;
}

extern "C" ovl_status eigsumr_accumulate(ovl_ctx* c, ovl_defl** defl, int n_eig, int m_basis, double mu,
                                         const void* rhs, void* x, int dtype, int on_device, double tol,
                                         ovl_solve_info* info) {
  OVL_TRY(check_io(c, rhs, x, 1, dtype));
  if (!defl) return set_err(c, OVL_EINVAL, "defl must not be null");
  if (n_eig < 1 || m_basis <= n_eig || m_basis > 1024) return set_err(c, OVL_EINVAL, "need 1 <= n_eig < m_basis <= 1024");
  if (!(mu > 0 && mu < 1)) return set_err(c, OVL_EINVAL, "mu must lie in (0, 1)");
  const int prec = c->P.mixed ? P32 : P64;
  ovl_defl* d = *defl;
  bool fresh = false;
  if (!d) {
    d = new (std::nothrow) ovl_defl();
    if (!d) return OVL_ENOMEM;
    fresh = true;
    ovl_status s = defl_alloc(c, d, prec, n_eig);
    if (s != OVL_OK) {
      ovl_defl_destroy(d);
      return s;
    }
  } else if (d->ctx != c) {
    return set_err(c, OVL_EINVAL, "deflation space belongs to another context");
  }
  // a space created here goes back on every error exit; only the last line hands it over
  struct FreshSpace {
    ovl_defl* d;
    bool own;
    ~FreshSpace() {
      if (own) ovl_defl_destroy(d);
    }
  } guard{d, fresh};
  EigState e;
  e.prec = d->v.prec;
  e.m = m_basis;
  e.n_eig = n_eig;
  e.mu = mu;
  e.delta = c->P.delta_split;
  OVL_TRY(get_field(c, "e_V", e.prec, m_basis, &e.V));
  OVL_TRY(get_field(c, "e_W", e.prec, m_basis, &e.W));
  if (!fresh && d->n > 0) {
    const int ns = std::min(d->n, n_eig);
    OVL_TRY(copy_convert(c, d->v, 0, *e.V, 0, ns));
    OVL_TRY(copy_convert(c, d->w, 0, *e.W, 0, ns));
    e.k = ns;
    e.n_seeded = ns;
  }
  // The accumulation rides on the context's middle solver: SUMR's Krylov basis (eigSUMR,
  // Alg. 5) or the residual directions of relCG (eigCG, Sec. 5); the space itself
  // (eigenvectors of D^dag D) serves both solvers.
  const bool use_cg = c->P.solver == OVL_SOLVER_CG;
  if (use_cg) {
    OVL_TRY(get_field(c, "e_Tp", e.prec, 1, &e.Tprev));
    OVL_TRY(get_field(c, "e_Zp", e.prec, 1, &e.Zprev));
  }
  EigHook hook;
  hook.active = true;
  hook.target = std::sqrt(tol);   // GMRESR in two steps while the eigenvectors are being calculated (Sec. 6)
  hook.eta_cap = e.eps_v;
  hook.hook = use_cg ? nullptr : eig_hook;
  hook.cg_hook = use_cg ? eig_cg_hook : nullptr;
  hook.after_outer = eig_after_outer;
  hook.data = &e;
  e.eig = &hook;
  Field *fb, *fx;
  OVL_TRY(get_field(c, "api_b", P64, 1, &fb));
  OVL_TRY(get_field(c, "bat_x", P64, 1, &fx));
  OVL_TRY(import_spinors(c, rhs, dtype, on_device, 1, *fb, 0));
  std::vector<double> mus(1, mu);
  // the deflation held so far accelerates this solve too; the space is rebuilt after it
  ovl_defl* use = (!fresh && d->n > 0) ? d : nullptr;
  ovl_status st = gmresr_batch(c, 1, mus, *fb, 0, *fx, 0, tol, use, info, &hook);
  if (st != OVL_OK && st != OVL_ENOCONV) return st;
  // final Ritz step over whatever the basis holds
  if (e.k > e.n_seeded || e.ndiag == 0 || e.k > n_eig) OVL_TRY(ritz_step(c, &e, n_eig));
  const int nk = e.k;
  if (nk < 1) return set_err(c, OVL_ENOCONV, "eigSUMR collected no basis vectors (the solve needed no SUMR step)");
  OVL_TRY(defl_store(c, d, e.V, nk, mu));
  OVL_TRY(export_spinors(c, x, dtype, on_device, 1, *fx, 0));
  if (info && c->P.verify) {
    std::vector<double> tr;
    OVL_TRY(true_residuals(c, *fb, 0, *fx, 0, 1, mus, tol, tr));
    info[0].true_residual = tr[0];
    info[0].converged = tr[0] <= tol * 1.0000001 ? 1 : 0;
  }
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  // the accumulation basis (4 x m_basis spinors) is not needed between solves
  for (const char* nm : {"e_V", "e_W", "e_VD", "e_T", "e_Tp", "e_Zp", "e_tmp"}) {
    auto it = c->ws.find(nm);
    if (it != c->ws.end()) free_field(it->second);
  }
  guard.own = false;
  *defl = d;
  return st;
}

extern "C" ovl_status ovl_ritz_recalculate(ovl_ctx* c, int m, int n_keep, double mu, double delta, const void* v,
                                           const void* vD, void* v_out, void* vD_out, int dtype, int on_device,
                                           double* ritz, double* residuals) {
  if (!c) return OVL_EINVAL;
  if (!v || !vD || !v_out || !vD_out || !ritz) return set_err(c, OVL_EINVAL, "null pointer");
  if (m < 1 || m > 1024 || n_keep < 1 || n_keep > m) return set_err(c, OVL_EINVAL, "need 1 <= n_keep <= m <= 1024");
  if (!(mu > 0 && mu < 1)) return set_err(c, OVL_EINVAL, "mu must lie in (0, 1)");
  if (dtype != OVL_C128 && dtype != OVL_C64) return set_err(c, OVL_EINVAL, "dtype must be OVL_C128 or OVL_C64");
  EigState e;
  e.prec = P64;
  e.m = m;
  e.n_eig = n_keep;
  e.mu = mu;
  e.delta = delta;
  Field* VD;
  OVL_TRY(get_field(c, "e_V", P64, m, &e.V));
  OVL_TRY(get_field(c, "e_W", P64, m, &e.W));
  OVL_TRY(get_field(c, "rr_vd", P64, m, &VD));
  OVL_TRY(import_spinors(c, v, dtype, on_device, m, *e.V, 0));
  OVL_TRY(import_spinors(c, vD, dtype, on_device, m, *VD, 0));
  // the basis keeps w with D v = (1+mu)/2 v + (1-mu)/2 w
  std::vector<cd> a(m, 2.0 / (1.0 - mu)), b(m, -(1.0 + mu) / (1.0 - mu));
  OVL_TRY(axpby_batch(c, a, *VD, 0, b, *e.V, 0, *e.W, 0, m));
  e.k = m;
  OVL_TRY(ritz_step(c, &e, n_keep, false));
  const int nk = e.k;
  if (nk < n_keep) return set_err(c, OVL_EBREAKDOWN, "the basis spans fewer than n_keep directions");
  std::vector<cd> av(n_keep, 0.5 * (1.0 - mu)), bv(n_keep, 0.5 * (1.0 + mu));
  OVL_TRY(axpby_batch(c, av, *e.W, 0, bv, *e.V, 0, *VD, 0, n_keep));
  OVL_TRY(export_spinors(c, v_out, dtype, on_device, n_keep, *e.V, 0));
  OVL_TRY(export_spinors(c, vD_out, dtype, on_device, n_keep, *VD, 0));
  for (int i = 0; i < n_keep; ++i) {
    ritz[i] = e.ritz[i];
    if (residuals) residuals[i] = e.res[i];
  }
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  return OVL_OK;
}

// Standalone eigensolver (Sec. 6): the eigSUMR Arnoldi process (Alg. 1 basis of
// V = gamma5 eps(K), accumulated by Algs. 5-6) run for its own sake, in rounds of
// `round_diags` Ritz steps. Each round ends with a Rayleigh-Ritz step over the current
// vectors and those of the previous two rounds, an accurate recomputation of v^D, and a
// restart from SUMR's last q orthogonalised against the current vectors; the sign
// accuracy follows the Sec. 5.1 bound that the Ritz step computes.
extern "C" ovl_status ovl_eigensolve(ovl_ctx* c, ovl_defl** defl, int n_eig, int m_basis, double mu,
                                     const void* start, int dtype, int on_device, int max_steps, double res_tol,
                                     int round_diags, int* steps_done) {
  if (!c) return OVL_EINVAL;
  if (!defl) return set_err(c, OVL_EINVAL, "defl must not be null");
  if (n_eig < 1 || m_basis < 2 * n_eig + 8 || m_basis > 1024)
    return set_err(c, OVL_EINVAL, "need n_eig >= 1 and 2 n_eig + 8 <= m_basis <= 1024");
  if (!(mu > 0 && mu < 1)) return set_err(c, OVL_EINVAL, "mu must lie in (0, 1)");
  if (max_steps < 1 || round_diags < 1) return set_err(c, OVL_EINVAL, "need max_steps >= 1 and round_diags >= 1");
  if (start && dtype != OVL_C128 && dtype != OVL_C64) return set_err(c, OVL_EINVAL, "bad dtype");
  const int prec = c->P.mixed ? P32 : P64;
  ovl_defl* d = *defl;
  bool fresh = false;
  if (!d) {
    d = new (std::nothrow) ovl_defl();
    if (!d) return OVL_ENOMEM;
    fresh = true;
    ovl_status s = defl_alloc(c, d, prec, n_eig);
    if (s != OVL_OK) {
      ovl_defl_destroy(d);
      return s;
    }
  } else if (d->ctx != c) {
    return set_err(c, OVL_EINVAL, "deflation space belongs to another context");
  } else if (d->cap < n_eig) {
    return set_err(c, OVL_EINVAL, "the space holds fewer than n_eig vectors");
  }
  auto fail = [&](ovl_status st) {
    if (fresh) ovl_defl_destroy(d);
    return st;
  };
  EigState e;
  e.prec = d->v.prec;
  e.m = m_basis;
  e.n_eig = n_eig;
  e.mu = mu;
  e.delta = c->P.delta_split;
  Field *q0, *xd, *g1v, *g1w, *g2v, *g2w;
  ovl_status st = OVL_OK;
  if ((st = get_field(c, "e_V", e.prec, m_basis, &e.V)) != OVL_OK) return fail(st);
  if ((st = get_field(c, "e_W", e.prec, m_basis, &e.W)) != OVL_OK) return fail(st);
  if ((st = get_field(c, "es_q0", e.prec, 1, &q0)) != OVL_OK) return fail(st);
  if ((st = get_field(c, "es_x", e.prec, 1, &xd)) != OVL_OK) return fail(st);
  if ((st = get_field(c, "es_g1v", e.prec, n_eig, &g1v)) != OVL_OK) return fail(st);
  if ((st = get_field(c, "es_g1w", e.prec, n_eig, &g1w)) != OVL_OK) return fail(st);
  if ((st = get_field(c, "es_g2v", e.prec, n_eig, &g2v)) != OVL_OK) return fail(st);
  if ((st = get_field(c, "es_g2w", e.prec, n_eig, &g2w)) != OVL_OK) return fail(st);
  // start vector: the caller's, or a Z2 source (every real component +-1, Sec. 6)
  if (start) {
    if ((st = import_spinors(c, start, dtype, on_device, 1, *q0, 0)) != OVL_OK) return fail(st);
  } else {
    std::vector<double> h((size_t)24 * c->V);
    unsigned long long r = 0x2545F4914F6CDD1Dull;
    for (auto& xv : h) {
      r ^= r << 13;
      r ^= r >> 7;
      r ^= r << 17;
      xv = (r >> 63) ? 1.0 : -1.0;
    }
    if ((st = import_spinors(c, h.data(), OVL_C128, 0, 1, *q0, 0)) != OVL_OK) return fail(st);
  }
  int n1 = 0, n2 = 0, total = 0;
  int ns = (!fresh && d->n > 0) ? std::min(d->n, n_eig) : 0;
  std::vector<double> mus(1, mu);
  for (int round = 0; total < max_steps; ++round) {
    // seed the basis with the current space; q0 orthogonalised against it
    e.k = 0;
    e.n_seeded = 0;
    e.ndiag = 0;
    if (ns > 0) {
      // the Gram blocks of the space (absent after ovl_defl_load until first use; n x n with
      // n = d->n, which exceeds ns when the caller's space holds more than n_eig vectors)
      if ((st = defl_prepare(c, d)) != OVL_OK) return fail(st);
      if ((st = copy_convert(c, d->v, 0, *e.V, 0, ns)) != OVL_OK) return fail(st);
      if ((st = copy_convert(c, d->w, 0, *e.W, 0, ns)) != OVL_OK) return fail(st);
      e.k = e.n_seeded = ns;
      for (int pass = 0; pass < 2; ++pass) {
        std::vector<cd> G, C;
        if ((st = gram_host(c, d->v, 0, ns, *q0, 0, 1, 0, G)) != OVL_OK) return fail(st);
        C.resize(ns);
        for (int i = 0; i < ns; ++i) C[i] = -G[i] / std::max(d->VV[(size_t)i * d->n + i].real(), 1e-300);
        if ((st = combine_host(c, d->v, 0, ns, C, *q0, 0, 1, 1)) != OVL_OK) return fail(st);
      }
    }
    SumrCfg cfg;
    cfg.prec = e.prec;
    cfg.target = 1e-300;   // no solve: the process runs for its basis alone
    cfg.floor = c->P.eta_floor;
    cfg.eta_dyn = &e.eta_cap;
    cfg.maxit = std::min(max_steps - total, (m_basis - e.k) + (round_diags - 1) * (m_basis - 2 * n_eig));
    cfg.qdrift = 0.1;
    cfg.hook = eig_hook;
    cfg.hook_data = &e;
    SumrResult sr;
    if ((st = sumr_batch(c, cfg, 1, mus, *q0, 0, *xd, 0, sr)) != OVL_OK) return fail(st);
    total += std::max(1, sr.sign_calls[0]);
    if (e.k > e.n_seeded || e.ndiag == 0) {
      if ((st = ritz_step(c, &e, n_eig)) != OVL_OK) return fail(st);
    }
    // Rayleigh-Ritz over this round's vectors and the previous two rounds'
    const int k0 = e.k;
    if (n1 > 0 && k0 + n1 + n2 <= m_basis) {
      if ((st = copy_convert(c, *g1v, 0, *e.V, k0, n1)) != OVL_OK) return fail(st);
      if ((st = copy_convert(c, *g1w, 0, *e.W, k0, n1)) != OVL_OK) return fail(st);
      if (n2 > 0) {
        if ((st = copy_convert(c, *g2v, 0, *e.V, k0 + n1, n2)) != OVL_OK) return fail(st);
        if ((st = copy_convert(c, *g2w, 0, *e.W, k0 + n1, n2)) != OVL_OK) return fail(st);
      }
      e.k = k0 + n1 + n2;
      e.n_seeded = 0;
      if ((st = ritz_step(c, &e, n_eig)) != OVL_OK) return fail(st);
    }
    ns = std::min(e.k, n_eig);
    if ((st = defl_store(c, d, e.V, ns, mu)) != OVL_OK) return fail(st);
    // generations: the previous round moves back, this one becomes the newest
    if (n1 > 0) {
      if ((st = copy_convert(c, *g1v, 0, *g2v, 0, n1)) != OVL_OK) return fail(st);
      if ((st = copy_convert(c, *g1w, 0, *g2w, 0, n1)) != OVL_OK) return fail(st);
    }
    n2 = n1;
    if ((st = copy_convert(c, d->v, 0, *g1v, 0, ns)) != OVL_OK) return fail(st);
    if ((st = copy_convert(c, d->w, 0, *g1w, 0, ns)) != OVL_OK) return fail(st);
    n1 = ns;
    double rmax = 0.0;
    for (int i = 0; i < ns; ++i) rmax = std::max(rmax, d->res[i]);
    if (ns >= n_eig && rmax <= res_tol) break;
    // restart from SUMR's last basis vector
    auto it = c->ws.find("s_q");
    if (it == c->ws.end()) break;
    if ((st = copy_convert(c, it->second, 0, *q0, 0, 1)) != OVL_OK) return fail(st);
  }
  {
    const cudaError_t ce = cudaStreamSynchronize(c->st);
    if (ce != cudaSuccess) return fail(cuda_check(c, ce, "cudaStreamSynchronize(c->st)"));
  }
  for (const char* nm : {"e_V", "e_W", "e_VD", "e_T", "es_q0", "es_x", "es_g1v", "es_g1w", "es_g2v", "es_g2w"}) {
    auto it = c->ws.find(nm);
    if (it != c->ws.end()) free_field(it->second);
  }
  if (steps_done) *steps_done = total;
  *defl = d;
  return OVL_OK;
}

extern "C" ovl_status ovl_defl_info(const ovl_defl* d, int* n, double* ritz, double* residuals) {
  if (!d) return OVL_EINVAL;
  if (n) *n = d->n;
  if (ritz) memcpy(ritz, d->ritz.data(), sizeof(double) * d->n);
  if (residuals) memcpy(residuals, d->res.data(), sizeof(double) * d->n);
  return OVL_OK;
}

extern "C" ovl_status ovl_defl_vector(const ovl_defl* d, int i, double* v, double* vD) {
  if (!d || i < 0 || i >= d->n) return OVL_EINVAL;
  ovl_ctx* c = d->ctx;
  if (v) OVL_TRY(export_spinors(c, v, OVL_C128, 0, 1, d->v, i));
  if (vD) {
    // v^D = (1+mu)/2 psi + (1-mu)/2 w at the space's mass
    Field* t;
    OVL_TRY(get_field(c, "dv_t", d->v.prec, 1, &t));
    std::vector<cd> a(1, 0.5 * (1.0 - d->mu)), b(1, 0.5 * (1.0 + d->mu));
    OVL_TRY(axpby_batch(c, a, d->w, i, b, d->v, i, *t, 0, 1));
    OVL_TRY(export_spinors(c, vD, OVL_C128, 0, 1, *t, 0));
  }
  return OVL_OK;
}

extern "C" ovl_status ovl_defl_save(const ovl_defl* d, const char* path) {
  if (!d || !path) return OVL_EINVAL;
  ovl_ctx* c = d->ctx;
  FILE* f = fopen(path, "wb");
  if (!f) return set_err(c, OVL_EINVAL, std::string("cannot open ") + path);
  // every write is checked: a full disk must not leave a truncated file reported as saved
  bool ok = fprintf(f, "OVLDEFL 1 n=%d V=%d mu=%.17g\n", d->n, c->V, d->mu) > 0;
  std::vector<double> h((size_t)24 * c->V);
  for (int i = 0; i < d->n && ok; ++i) {
    ovl_status s = export_spinors(c, h.data(), OVL_C128, 0, 1, d->v, i);
    if (s != OVL_OK) { fclose(f); return s; }
    ok = fwrite(h.data(), sizeof(double), h.size(), f) == h.size();
    s = export_spinors(c, h.data(), OVL_C128, 0, 1, d->w, i);
    if (s != OVL_OK) { fclose(f); return s; }
    ok = ok && fwrite(h.data(), sizeof(double), h.size(), f) == h.size();
  }
  ok = ok && fwrite(d->ritz.data(), sizeof(double), d->n, f) == (size_t)d->n;
  ok = ok && fwrite(d->res.data(), sizeof(double), d->n, f) == (size_t)d->n;
  ok = (fclose(f) == 0) && ok;
  if (!ok) return set_err(c, OVL_EINVAL, std::string("writing ") + path + " failed");
  return OVL_OK;
}

extern "C" ovl_status ovl_defl_load(ovl_ctx* c, ovl_defl** out, const char* path) {
  if (!c || !out || !path) return OVL_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return set_err(c, OVL_EINVAL, std::string("cannot open ") + path);
  int n = 0, V = 0;
  double mu = 0;
  if (fscanf(f, "OVLDEFL 1 n=%d V=%d mu=%lf", &n, &V, &mu) != 3 || fgetc(f) != '\n' || V != c->V || n < 0) {
    fclose(f);
    return set_err(c, OVL_EINVAL, "bad deflation file header");
  }
  ovl_defl* d = new (std::nothrow) ovl_defl();
  if (!d) { fclose(f); return OVL_ENOMEM; }
  ovl_status s = defl_alloc(c, d, c->P.mixed ? P32 : P64, std::max(n, 1));
  std::vector<double> h((size_t)24 * c->V);
  for (int i = 0; i < n && s == OVL_OK; ++i) {
    if (fread(h.data(), sizeof(double), h.size(), f) != h.size()) s = set_err(c, OVL_EINVAL, "short file");
    else s = import_spinors(c, h.data(), OVL_C128, 0, 1, d->v, i);
    if (s != OVL_OK) break;
    if (fread(h.data(), sizeof(double), h.size(), f) != h.size()) s = set_err(c, OVL_EINVAL, "short file");
    else s = import_spinors(c, h.data(), OVL_C128, 0, 1, d->w, i);
  }
  d->ritz.assign(n, 0.0);
  d->res.assign(n, 0.0);
  if (s == OVL_OK && n > 0) {
    if (fread(d->ritz.data(), sizeof(double), n, f) != (size_t)n || fread(d->res.data(), sizeof(double), n, f) != (size_t)n)
      s = set_err(c, OVL_EINVAL, "short file");
  }
  fclose(f);
  if (s != OVL_OK) {
    ovl_defl_destroy(d);
    return s;
  }
  d->n = n;
  d->mu = mu;
  cudaStreamSynchronize(c->st);
  *out = d;
  return OVL_OK;
}

// ---------------------------------------------------------------- force
extern "C" ovl_status overlap_force(ovl_ctx* c, double mu, const void* phi, int dtype, int on_device, double tol,
                                    double* dSdU, double* S) {
  if (!c || !phi || !dSdU) return OVL_EINVAL;
  if (!(mu > 0 && mu < 1)) return set_err(c, OVL_EINVAL, "mu must lie in (0, 1)");
  if (c->kd_n > 0)
    return set_err(c, OVL_EINVAL,
                   "overlap_force differentiates the Zolotarev rational itself: remove the kernel low-mode "
                   "deflation first (ovl_kernel_deflate with n_ev = 0)");
  Field* fp;
  OVL_TRY(get_field(c, "f_phi", P64, 1, &fp));
  OVL_TRY(import_spinors(c, phi, dtype, on_device, 1, *fp, 0));
  return force_compute(c, mu, *fp, tol, dSdU, S);
}

// ---------------------------------------------------------------- profiling
extern "C" ovl_status ovl_profile_enable(ovl_ctx* c, int on) {
  if (!c) return OVL_EINVAL;
  if (!on) prof_flush(c);
  c->prof.on = on != 0;
  return OVL_OK;
}
extern "C" ovl_status ovl_profile_reset(ovl_ctx* c) {
  if (!c) return OVL_EINVAL;
  prof_flush(c);
  for (int k = 0; k < OVL_PROF_CLASSES; ++k) {
    c->prof.launches[k] = 0;
    c->prof.ms[k] = 0;
    c->prof.bytes[k] = 0;
    c->prof.units[k] = 0;
  }
  c->wcalls[0] = c->wcalls[1] = c->wcalls[2] = 0;
  return OVL_OK;
}
extern "C" ovl_status ovl_profile_get(ovl_ctx* c, int cls, long long* launches, double* ms, double* bytes) {
  if (!c || cls < 0 || cls >= OVL_PROF_CLASSES) return OVL_EINVAL;
  prof_flush(c);
  if (launches) *launches = c->prof.launches[cls];
  if (ms) *ms = c->prof.ms[cls];
  if (bytes) *bytes = c->prof.bytes[cls];
  return OVL_OK;
}

extern "C" ovl_status ovl_wilson_tuning(const ovl_ctx* c, int prec, int* variant, double* ms0, double* ms1,
                                        double* ms2, double* ms3) {
  if (!c || prec < P64 || prec > P64E) return OVL_EINVAL;
  if (variant) *variant = c->wvar[prec];
  if (ms0) *ms0 = c->wtime[prec][0];
  if (ms1) *ms1 = c->wtime[prec][1];
  if (ms2) *ms2 = c->wtime[prec][2];
  if (ms3) *ms3 = c->wtime[prec][3];
  return OVL_OK;
}

extern "C" ovl_status ovl_profile_units(ovl_ctx* c, int cls, double* units) {
  if (!c || cls < 0 || cls >= OVL_PROF_CLASSES || !units) return OVL_EINVAL;
  prof_flush(c);
  *units = c->prof.units[cls];
  return OVL_OK;
}

extern "C" ovl_status ovl_bench_wilson(ovl_ctx* c, int prec, int n, int iters, double* ms_per_launch,
                                       double* bytes_per_launch) {
  if (!c || prec < P64 || prec > P64E || n < 1 || n > 256 || iters < 1) return OVL_EINVAL;
  Field *fi, *fo;
  OVL_TRY(get_field(c, "bw_in", prec, n, &fi));
  OVL_TRY(get_field(c, "bw_out", prec, n, &fo));
  {
    std::vector<double> h((size_t)24 * c->V);
    unsigned long long st = 12345;
    for (auto& x : h) {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      x = ((double)(st >> 11) / 9007199254740992.0) - 0.5;
    }
    for (int j = 0; j < n; ++j) OVL_TRY(import_spinors(c, h.data(), OVL_C128, 0, 1, *fi, j));
  }
  for (int w = 0; w < 3; ++w) OVL_TRY(wilson_apply_field(c, prec, *fi, 0, *fo, 0, n));
  cudaEvent_t e0, e1;
  OVL_CUDA(c, cudaEventCreate(&e0));
  OVL_CUDA(c, cudaEventCreate(&e1));
  OVL_CUDA(c, cudaEventRecord(e0, c->st));
  for (int k = 0; k < iters; ++k) launch_wilson_K(prec, prec, prec, c->g, c->kappa, links_of(c, prec), fi->ref(), fo->ref(), n, nullptr, nullptr, c->st);
  OVL_CUDA(c, cudaEventRecord(e1, c->st));
  OVL_CUDA(c, cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  OVL_TRY(check_launch(c, __func__));
  const double sb = prec == P16 ? 52 : spinor_site_bytes(prec);
  const double lb = prec == P64E ? 576 : prec == P64 ? 384 : prec == P32 ? 192 : 96;   // algorithmic
  if (ms_per_launch) *ms_per_launch = ms / iters;
  if (bytes_per_launch) *bytes_per_launch = (double)c->V * (2.0 * sb * n + lb);
  return OVL_OK;
}

// ---------------------------------------------------------------- dense Gram block
extern "C" ovl_status ovl_gram(ovl_ctx* c, const void* A, int na, const void* B, int nb, int dtype, int on_device,
                               int prec, int g5, int method, double* G) {
  if (!c) return OVL_EINVAL;
  if (!A || !B || !G) return set_err(c, OVL_EINVAL, "null pointer");
  if (na < 1 || na > 1024 || nb < 1 || nb > 1024) return set_err(c, OVL_EINVAL, "na and nb must lie in 1..1024");
  if (dtype != OVL_C128 && dtype != OVL_C64) return set_err(c, OVL_EINVAL, "dtype must be OVL_C128 or OVL_C64");
  if (prec != P64 && prec != P32) return set_err(c, OVL_EINVAL, "prec must be OVL_PREC_F64 or OVL_PREC_F32");
  if (method != 0 && method != 1) return set_err(c, OVL_EINVAL, "method must be 0 or 1");
  Field *fa, *fb;
  OVL_TRY(get_field(c, "gr_a", prec, na, &fa));
  OVL_TRY(get_field(c, "gr_b", prec, nb, &fb));
  OVL_TRY(import_spinors(c, A, dtype, on_device, na, *fa, 0));
  OVL_TRY(import_spinors(c, B, dtype, on_device, nb, *fb, 0));
  const int saved = c->P.gram_method;
  c->P.gram_method = method;
  std::vector<cd> Gh;
  const ovl_status st = gram_host(c, *fa, 0, na, *fb, 0, nb, g5 ? 1 : 0, Gh);
  c->P.gram_method = saved;
  if (st != OVL_OK) return st;
  for (size_t k = 0; k < Gh.size(); ++k) {
    G[2 * k] = Gh[k].real();
    G[2 * k + 1] = Gh[k].imag();
  }
  return OVL_OK;
}

extern "C" ovl_status ovl_bench_gram(ovl_ctx* c, int prec, int na, int nb, int method, int iters, double* ms_per_call) {
  if (!c || (prec != P64 && prec != P32) || na < 1 || na > 1024 || nb < 1 || nb > 1024 || iters < 1 ||
      (method != 0 && method != 1) || !ms_per_call)
    return OVL_EINVAL;
  Field *fa, *fb;
  OVL_TRY(get_field(c, "bg_a", prec, na, &fa));
  OVL_TRY(get_field(c, "bg_b", prec, nb, &fb));
  {
    std::vector<double> h((size_t)24 * c->V);
    unsigned long long st = 6789;
    for (int j = 0; j < na + nb; ++j) {
      for (auto& x : h) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        x = ((double)(st >> 11) / 9007199254740992.0) - 0.5;
      }
      OVL_TRY(import_spinors(c, h.data(), OVL_C128, 0, 1, j < na ? *fa : *fb, j < na ? j : j - na));
    }
  }
  const int saved = c->P.gram_method;
  c->P.gram_method = method;
  double* dG = nullptr;
  int* derr = nullptr;
  ovl_status s = gram_device(c, *fa, 0, na, *fb, 0, nb, 0, &dG, &derr);   // sizes the work buffer
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (s == OVL_OK && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    cudaEventRecord(e0, c->st);
    for (int k = 0; k < iters && s == OVL_OK; ++k) s = gram_device(c, *fa, 0, na, *fb, 0, nb, 0, &dG, &derr);
    cudaEventRecord(e1, c->st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_per_call = ms / iters;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->P.gram_method = saved;
  OVL_TRY(s);
  int herr = 0;
  if (derr) OVL_CUDA(c, cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) return set_err(c, OVL_ETIMEOUT, "tensor-core Gram block: a bounded wait on the MMA pipeline gave up");
  return OVL_OK;
}

// ---------------------------------------------------------------- FP32 issue probe
namespace ovl {
void launch_fma_probe(int nblocks, int iters, float* out, cudaStream_t st);
}
extern "C" ovl_status ovl_bench_fp32(ovl_ctx* c, double* fma_per_s) {
  if (!c || !fma_per_s) return OVL_EINVAL;
  int nsm = 0;
  OVL_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  const int nblocks = nsm * 8, iters = 4096;
  float* d = nullptr;
  OVL_CUDA(c, cudaMalloc((void**)&d, sizeof(float) * nblocks * 256));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch_fma_probe(nblocks, iters, d, c->st);
  cudaEventRecord(e0, c->st);
  const int reps = 20;
  for (int r = 0; r < reps; ++r) launch_fma_probe(nblocks, iters, d, c->st);
  cudaEventRecord(e1, c->st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (err != cudaSuccess) return cuda_check(c, err, "ovl_bench_fp32");
  OVL_TRY(check_launch(c, __func__));
  // 8 independent FMA chains of `iters` steps per thread, 256 threads per block
  *fma_per_s = (double)reps * nblocks * 256.0 * 8.0 * iters / (ms * 1e-3);
  return OVL_OK;
}
