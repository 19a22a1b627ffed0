// Context, workspaces, caller I/O, profiling and the sign-function driver of
// liboverlap. The sign function (Sec. 3) is
//   eps(K) v = sum_i omega_i K (K^2 + sigma_i)^-1 v,
// evaluated by the device-resident multi-shift CG of mscg.cu; this file runs its
// host loop: a chunk of steps is issued without synchronising, then one small
// copy of the per-system done flags decides whether another chunk is needed.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "context.h"
#include "hostmath.h"
#include "solver.h"

namespace ovl {

ovl_status set_err(ovl_ctx* c, ovl_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

ovl_status cuda_check(ovl_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string("CUDA error ") + cudaGetErrorString(e) + " in " + what;
  return set_err(c, OVL_ECUDA, m);
}

static thread_local bool g_bad_combo = false;
static thread_local const char* g_bad_where = "";
void note_bad_combo(const char* where) {
  g_bad_combo = true;
  g_bad_where = where;
}
bool take_bad_combo() {
  const bool b = g_bad_combo;
  g_bad_combo = false;
  return b;
}

ovl_status check_launch(ovl_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, where);
  if (take_bad_combo())
    return set_err(c, OVL_EINVAL, std::string("unsupported precision combination in ") + g_bad_where + " (" + where + ")");
  return OVL_OK;
}

static size_t spinor_bytes(int prec) { return (size_t)spinor_site_bytes(prec); }

void free_field(Field& f) {
  if (f.data) cudaFree(f.data);
  if (f.norm) cudaFree(f.norm);
  f.data = nullptr;
  f.norm = nullptr;
  f.n = 0;
}

ovl_status get_field(ovl_ctx* c, const std::string& name, int prec, int n, Field** out) {
  Field& f = c->ws[name];
  if (f.data != nullptr && f.prec == prec && f.n >= n) {
    *out = &f;
    return OVL_OK;
  }
  if (f.data != nullptr) {
    cudaStreamSynchronize(c->st);
    free_field(f);
  }
  f.prec = prec;
  f.V = c->V;
  f.n = n;
  const size_t bytes = spinor_bytes(prec) * (size_t)c->V * n;
  if (cudaMalloc(&f.data, bytes) != cudaSuccess) {
    cudaGetLastError();
    f.data = nullptr;
    // the stored Lanczos basis is a cache sized from the free memory: give it back (and
    // the graphs that point into it) unless a sign application is using it right now
    if (c->lz_pool && !c->lz_pool_busy) {
      cudaStreamSynchronize(c->st);
      cudaFree(c->lz_pool);
      c->lz_pool = nullptr;
      c->lz_pool_bytes = 0;
      for (auto& g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
      c->graphs.clear();
      if (cudaMalloc(&f.data, bytes) != cudaSuccess) {
        cudaGetLastError();
        f.data = nullptr;
      }
    }
  }
  if (f.data == nullptr) {
    f.n = 0;
    return set_err(c, OVL_ENOMEM, "cudaMalloc failed for workspace " + name);
  }
  if (prec == P16) {
    if (cudaMalloc((void**)&f.norm, sizeof(float) * (size_t)c->V * n) != cudaSuccess) {
      cudaGetLastError();
      free_field(f);
      return set_err(c, OVL_ENOMEM, "cudaMalloc failed for workspace norms " + name);
    }
  }
  *out = &f;
  return OVL_OK;
}

ovl_status ensure_partials(ovl_ctx* c, int nrhs) {
  const size_t need = (size_t)nrhs * ((c->V + BX - 1) / BX) * NVRED;
  if (need <= c->partials_n) return OVL_OK;
  if (c->partials) {
    cudaStreamSynchronize(c->st);
    cudaFree(c->partials);
  }
  OVL_CUDA(c, cudaMalloc((void**)&c->partials, need * sizeof(double)));
  c->partials_n = need;
  return OVL_OK;
}

ovl_status ensure_ms(ovl_ctx* c, int nrhs) {
  if (nrhs <= c->ms_n) return OVL_OK;
  if (c->ms) {
    cudaStreamSynchronize(c->st);
    cudaFree(c->ms);
  }
  OVL_CUDA(c, cudaMalloc((void**)&c->ms, sizeof(MsRhs) * nrhs));
  c->ms_n = nrhs;
  return OVL_OK;
}

ovl_status ensure_lz(ovl_ctx* c, int nrhs, int cap) {
  if (nrhs <= c->lz_n && cap <= c->lz_cap) return OVL_OK;
  const int n = std::max(nrhs, c->lz_n), k = std::max(cap, c->lz_cap);
  cudaStreamSynchronize(c->st);
  if (c->lz) cudaFree(c->lz);
  if (c->lz_hist) cudaFree(c->lz_hist);
  if (c->lz_Y) cudaFree(c->lz_Y);
  if (c->lz_coefW) cudaFree(c->lz_coefW);
  if (c->lz_ctr) cudaFree(c->lz_ctr);
  c->lz = nullptr;
  c->lz_hist = c->lz_Y = c->lz_coefW = nullptr;
  c->lz_ctr = nullptr;
  c->lz_n = c->lz_cap = 0;
  OVL_CUDA(c, cudaMalloc((void**)&c->lz, sizeof(LzRhs) * n));
  OVL_CUDA(c, cudaMalloc((void**)&c->lz_ctr, sizeof(unsigned int) * n));
  OVL_CUDA(c, cudaMemsetAsync(c->lz_ctr, 0, sizeof(unsigned int) * n, c->st));
  OVL_CUDA(c, cudaMalloc((void**)&c->lz_hist, sizeof(double) * 2 * (size_t)n * k));
  // sized for the largest pole count (kernel deflation can change the count later)
  OVL_CUDA(c, cudaMalloc((void**)&c->lz_Y, sizeof(double) * (size_t)n * NPMAX * 2 * k));
  OVL_CUDA(c, cudaMalloc((void**)&c->lz_coefW, sizeof(double) * (size_t)n * k));
  c->lz_n = n;
  c->lz_cap = k;
  return OVL_OK;
}

ovl_status lz_pool_field(ovl_ctx* c, int prec, int n, Field* out) {
  const size_t data = (size_t)spinor_bytes(prec) * c->V * n;
  const size_t norms = prec == P16 ? sizeof(float) * (size_t)c->V * n : 0;
  const size_t need = data + norms;
  if (need > c->lz_pool_bytes) {
    cudaStreamSynchronize(c->st);
    if (c->lz_pool) cudaFree(c->lz_pool);
    c->lz_pool = nullptr;
    c->lz_pool_bytes = 0;
    if (cudaMalloc(&c->lz_pool, need) != cudaSuccess) {
      cudaGetLastError();
      c->lz_pool = nullptr;
      return set_err(c, OVL_ENOMEM, "cudaMalloc failed for the stored Lanczos basis");
    }
    c->lz_pool_bytes = need;
  }
  out->prec = prec;
  out->n = n;
  out->V = c->V;
  out->data = c->lz_pool;
  out->norm = prec == P16 ? reinterpret_cast<float*>(static_cast<char*>(c->lz_pool) + data) : nullptr;
  return OVL_OK;
}

void trim_workspaces(ovl_ctx* c) {
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  for (auto& kv : c->ws) free_field(kv.second);
  c->ws.clear();
  if (c->lz_pool) cudaFree(c->lz_pool);
  c->lz_pool = nullptr;
  c->lz_pool_bytes = 0;
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

ovl_status ensure_stage(ovl_ctx* c, size_t bytes) {
  if (bytes <= c->hstage_bytes) return OVL_OK;
  // the last copy out of the old buffer must be done before it goes back
  if (c->hstage) OVL_CUDA(c, cudaEventSynchronize(c->stage_ev));
  if (c->hstage) cudaFreeHost(c->hstage);
  c->hstage = nullptr;
  OVL_CUDA(c, cudaMallocHost(&c->hstage, bytes));
  c->hstage_bytes = bytes;
  return OVL_OK;
}

ovl_status ensure_work(ovl_ctx* c, size_t nd) {
  if (nd <= c->dwork_n) return OVL_OK;
  if (c->dwork) {
    cudaStreamSynchronize(c->st);
    cudaFree(c->dwork);
  }
  OVL_CUDA(c, cudaMalloc((void**)&c->dwork, nd * sizeof(double)));
  c->dwork_n = nd;
  return OVL_OK;
}

LinkRef links_of(const ovl_ctx* c, int prec) {
  LinkRef r;
  r.data = c->link[prec];
  r.V = c->V;
  r.variant = c->wvar[prec];
  r.variant_multi = c->wvar_multi[prec];
  return r;
}

// ---------------------------------------------------------------- profiling
void prof_begin(ovl_ctx* c, int cls, ProfPair* p) {
  p->cls = cls;
  if (!c->prof.on) return;
  if (c->prof.pool.size() < 2) {
    for (int k = 0; k < 256; ++k) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->prof.pool.push_back(e);
    }
  }
  p->a = c->prof.pool.back();
  c->prof.pool.pop_back();
  p->b = c->prof.pool.back();
  c->prof.pool.pop_back();
  cudaEventRecord(p->a, c->st);
}

void prof_end(ovl_ctx* c, ProfPair* p, double bytes) {
  if (!c->prof.on) return;
  cudaEventRecord(p->b, c->st);
  p->bytes = bytes;
  c->prof.pending.push_back(*p);
  if (c->prof.pending.size() > 4096) prof_flush(c);
}

void prof_flush(ovl_ctx* c) {
  if (c->prof.pending.empty()) return;
  cudaEventSynchronize(c->prof.pending.back().b);
  for (auto& q : c->prof.pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, q.a, q.b);
    c->prof.launches[q.cls] += 1;
    c->prof.ms[q.cls] += ms;
    c->prof.bytes[q.cls] += q.bytes;
    c->prof.pool.push_back(q.a);
    c->prof.pool.push_back(q.b);
  }
  c->prof.pending.clear();
}

ovl_status upload(ovl_ctx* c, const double* host, int count, const double** dev) {
  const size_t lo = 32768, hi = 64 * 4096;
  if ((size_t)count > hi - lo) return set_err(c, OVL_EINVAL, "scalar upload too large");
  if (c->ring_pos < lo || c->ring_pos + count > hi) {
    // wrapping: every earlier upload and every kernel reading it must have finished
    OVL_CUDA(c, cudaStreamSynchronize(c->st));
    c->ring_pos = lo;
  }
  double* h = c->hpin + c->ring_pos;
  double* d = c->dscal + c->ring_pos;
  memcpy(h, host, sizeof(double) * count);
  OVL_CUDA(c, cudaMemcpyAsync(d, h, sizeof(double) * count, cudaMemcpyHostToDevice, c->st));
  c->ring_pos += (count + 31) & ~(size_t)31;
  *dev = d;
  return OVL_OK;
}

ovl_status wilson_apply_field(ovl_ctx* c, int prec, const Field& in, int ioff, Field& out, int ooff, int n) {
  launch_wilson_K(in.prec, prec, out.prec, c->g, c->kappa, links_of(c, prec), in.ref(ioff), out.ref(ooff), n, nullptr,
                  nullptr, c->st);
  OVL_TRY(check_launch(c, __func__));
  c->wcalls[prec] += n;
  return OVL_OK;
}

// ---------------------------------------------------------------- reductions
ovl_status reduce_to_host_nv(ovl_ctx* c, int nsb, int nrhs, double* out, int nv) {
  launch_reduce_partials(c->partials, nsb, nrhs, c->dred, c->st);
  double* h = c->hpin + 16384;   // NVRED * 4096 doubles
  OVL_CUDA(c, cudaMemcpyAsync(h, c->dred, sizeof(double) * NVRED * nrhs, cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  for (int j = 0; j < nrhs; ++j)
    for (int k = 0; k < nv; ++k) out[nv * j + k] = h[NVRED * j + k];
  return OVL_OK;
}

ovl_status reduce_to_host(ovl_ctx* c, int nsb, int nrhs, double* host_pairs) {
  return reduce_to_host_nv(c, nsb, nrhs, host_pairs, 2);
}

// ---------------------------------------------------------------- caller I/O
// Host buffers that are page-locked (cudaHostAlloc, cudaHostRegister, a pinned torch
// tensor) are copied by DMA directly; pageable ones go through the context's pinned
// staging buffer (one host memcpy each way).
static bool host_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

ovl_status import_spinors(ovl_ctx* c, const void* src, int dtype, int on_device, int n, Field& dst, int off) {
  const size_t esz = dtype == OVL_C128 ? 16 : 8;
  const size_t bytes = esz * 12 * (size_t)c->V * n;
  const void* dsrc = src;
  Field* tmp = nullptr;
  if (!on_device) {
    OVL_TRY(get_field(c, "io_canon", P64, (int)((bytes + 192 * (size_t)c->V - 1) / (192 * (size_t)c->V)), &tmp));
    if (host_pinned(src)) {
      OVL_CUDA(c, cudaMemcpyAsync(tmp->data, src, bytes, cudaMemcpyHostToDevice, c->st));
    } else {
      OVL_TRY(ensure_stage(c, bytes));
      // the previous copy out of the pinned staging buffer must have finished before it
      // is overwritten
      OVL_CUDA(c, cudaEventSynchronize(c->stage_ev));
      memcpy(c->hstage, src, bytes);
      OVL_CUDA(c, cudaMemcpyAsync(tmp->data, c->hstage, bytes, cudaMemcpyHostToDevice, c->st));
      OVL_CUDA(c, cudaEventRecord(c->stage_ev, c->st));
    }
    dsrc = tmp->data;
  }
  ProfPair pp;
  prof_begin(c, 4, &pp);
  launch_pack(dtype, dsrc, dst.prec, dst.ref(off), n, c->V, c->st);
  prof_end(c, &pp, (double)bytes + (double)n * c->V * spinor_bytes(dst.prec));
  OVL_TRY(check_launch(c, __func__));
  return OVL_OK;
}

ovl_status export_spinors(ovl_ctx* c, void* dst, int dtype, int on_device, int n, const Field& src, int off) {
  const size_t esz = dtype == OVL_C128 ? 16 : 8;
  const size_t bytes = esz * 12 * (size_t)c->V * n;
  if (on_device) {
    ProfPair pp;
    prof_begin(c, 4, &pp);
    launch_unpack(dtype, dst, src.prec, src.ref(off), n, c->V, c->st);
    prof_end(c, &pp, (double)bytes + (double)n * c->V * spinor_bytes(src.prec));
    OVL_TRY(check_launch(c, __func__));
    return OVL_OK;
  }
  Field* tmp = nullptr;
  OVL_TRY(get_field(c, "io_canon", P64, (int)((bytes + 192 * (size_t)c->V - 1) / (192 * (size_t)c->V)), &tmp));
  const bool pinned = host_pinned(dst);
  if (!pinned) OVL_TRY(ensure_stage(c, bytes));
  ProfPair pp;
  prof_begin(c, 4, &pp);
  launch_unpack(dtype, tmp->data, src.prec, src.ref(off), n, c->V, c->st);
  prof_end(c, &pp, (double)bytes + (double)n * c->V * spinor_bytes(src.prec));
  OVL_CUDA(c, cudaMemcpyAsync(pinned ? dst : c->hstage, tmp->data, bytes, cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  if (!pinned) memcpy(dst, c->hstage, bytes);
  return OVL_OK;
}

// ---------------------------------------------------------------- sign function
int choose_mode(const ovl_ctx* c, double eta) {
  const int accurate = c->P.emulate_fp64 ? SIGN64E : SIGN64;
  if (!c->P.mixed) return accurate;
  if (c->P.half_storage && eta >= c->P.half_switch) return SIGN16;
  if (eta >= c->P.sp_switch) return SIGN32;
  return accurate;
}

// Find or capture the cached graph for key. capture(stream) issues the launches; they
// are recorded on the context's private capture stream and instantiated once. At most
// kMaxGraphs graphs are kept (least recently used dropped).
static constexpr int kGraphIters = 8;
static constexpr int kLzCapMax = 1024;   // basis slots per Lanczos cycle (coefficient buffers)
static constexpr size_t kMaxGraphs = 16;
template <typename F>
static ovl_status ms_graph(ovl_ctx* c, const std::vector<unsigned long long>& key, cudaGraphExec_t* out, F capture) {
  ++c->graph_clock;
  for (auto& g : c->graphs)
    if (g.key == key) {
      g.last_use = c->graph_clock;
      *out = g.exec;
      return OVL_OK;
    }
  // the capture stream must not start before the work already queued on the context
  // stream that the graph will follow: graphs are launched on the context stream, so
  // capturing itself needs no ordering, only launches do.
  OVL_CUDA(c, cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal));
  capture(c->cap_st);
  cudaGraph_t graph = nullptr;
  const cudaError_t e1 = cudaStreamEndCapture(c->cap_st, &graph);
  OVL_TRY(check_launch(c, "multi-shift CG graph capture"));
  if (e1 != cudaSuccess) return cuda_check(c, e1, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return cuda_check(c, e2, "cudaGraphInstantiate");
  if (c->graphs.size() >= kMaxGraphs) {
    size_t old = 0;
    for (size_t i = 1; i < c->graphs.size(); ++i)
      if (c->graphs[i].last_use < c->graphs[old].last_use) old = i;
    cudaGraphExecDestroy(c->graphs[old].exec);
    c->graphs.erase(c->graphs.begin() + old);
  }
  MsGraph g;
  g.key = key;
  g.exec = exec;
  g.last_use = c->graph_clock;
  c->graphs.push_back(g);
  *out = exec;
  return OVL_OK;
}

static ovl_status sign_op_batch(ovl_ctx* c, int mode, const Field& v, int voff, Field& out, int ooff, int n,
                                const double* eta, double c1, double c2, const double* coef, int herm,
                                const Field* dot_w, int woff, double* dots, SignStats* stats);
static ovl_status sign_op_batch_lz(ovl_ctx* c, int mode, const Field& v, int voff, Field& out, int ooff, int n,
                                   const double* eta, double c1, double c2, const double* coef, int herm,
                                   const Field* dot_w, int woff, double* dots, SignStats* stats, int cap);

// decade of a sign accuracy, the key of the step-count memory
static int eta_decade(double e) {
  const int d = (int)std::floor(-std::log10(std::max(e, 1e-16)));
  return std::min(16, std::max(0, d));
}

// Basis slots for one stored-basis Lanczos cycle: the most steps this context has needed
// at this mode and accuracy, else the CG bound 1/2 sqrt(kappa) ln(2 N_Z / eta) for the
// base shift (kappa = (b^2 + sigma_0) / (a^2 + sigma_0)), with a quarter's margin.
static int lz_cap_for(const ovl_ctx* c, int mode, double eta) {
  if (c->P.lanczos_cap > 0) return c->P.lanczos_cap;
  const double s0 = c->hpoles.sigma0;
  const double kap = (c->zb * c->zb + s0) / (c->za * c->za + s0);
  int k = c->lz_kmax[mode][eta_decade(eta)];
  if (k <= 0) k = (int)std::ceil(0.5 * std::sqrt(kap) * std::log(2.0 * c->npoles / std::max(eta, 1e-16))) + 10;
  k = (int)std::ceil(1.25 * k) + 8;
  return std::max(16, std::min(std::min(k, c->P.mscg_max + 2), kLzCapMax));
}

// Systems per multi-shift solve are capped so that the pole vectors of one batch stay
// within kPoleBytes (24 poles x 36 systems of 24^3 x 48 in double-float would be 110 GB);
// larger requests run as consecutive sub-batches. The stored-basis Lanczos form is
// sub-batched so that cap basis vectors per system fit in params.basis_gb.
static constexpr double kPoleBytes = 64e9;
ovl_status sign_op(ovl_ctx* c, int mode, const Field& v, int voff, Field& out, int ooff, int n, const double* eta,
                   double c1, double c2, const double* coef, int herm, const Field* dot_w, int woff, double* dots,
                   SignStats* stats) {
  if (n <= 0) return OVL_OK;
  const int PP = mode == SIGN64 ? P64 : mode == SIGN32 ? P32 : mode == SIGN16 ? P16 : P64E;
  double emin = 1e300;
  for (int j = 0; j < n; ++j) emin = std::min(emin, eta[j] > 0 ? eta[j] : c->eps_sign);
  if (!c->exact_rational) emin = std::max(emin, c->delta);
  const int cap = lz_cap_for(c, mode, emin);
  const double per_lz = (double)cap * c->V * (spinor_bytes(PP) + (PP == P16 ? 4.0 : 0.0));
  // the basis budget: params.basis_gb, and never more than 70% of what the device has free
  // (counting the pool this context already holds); the rest is left to the workspaces of
  // the solvers around the sign, and a workspace that still does not fit takes the pool back
  double budget = c->P.basis_gb * 1e9;
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) budget = std::min(budget, 0.7 * ((double)fr + c->lz_pool_bytes));
    else cudaGetLastError();
  }
  const int n_fit = (int)std::min(1e9, budget / per_lz);
  const bool use_lz = c->P.sign_method == 2 || (c->P.sign_method == 0 && n_fit >= std::min(n, c->P.batch_max));
  if (use_lz) {
    const int nb = std::max(1, std::min(c->P.batch_max, n_fit));
    if (stats) {
      stats->iters.clear();
      stats->status.clear();
    }
    for (int j0 = 0; j0 < n; j0 += nb) {
      const int m = std::min(nb, n - j0);
      SignStats sub;
      OVL_TRY(sign_op_batch_lz(c, mode, v, voff + j0, out, ooff + j0, m, eta + j0, c1, c2,
                               coef ? coef + 2 * j0 : nullptr, herm, dot_w, woff + j0, dots ? dots + 4 * j0 : nullptr,
                               stats ? &sub : nullptr, cap));
      if (stats) {
        stats->iters.insert(stats->iters.end(), sub.iters.begin(), sub.iters.end());
        stats->status.insert(stats->status.end(), sub.status.begin(), sub.status.end());
      }
    }
    return OVL_OK;
  }
  const double per = (double)c->npoles * c->V * spinor_bytes(PP);
  int nb = std::max(1, std::min(c->P.batch_max, (int)(kPoleBytes / per)));
  if (n <= nb) return sign_op_batch(c, mode, v, voff, out, ooff, n, eta, c1, c2, coef, herm, dot_w, woff, dots, stats);
  if (stats) {
    stats->iters.clear();
    stats->status.clear();
  }
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int m = std::min(nb, n - j0);
    SignStats sub;
    OVL_TRY(sign_op_batch(c, mode, v, voff + j0, out, ooff + j0, m, eta + j0, c1, c2, coef ? coef + 2 * j0 : nullptr,
                          herm, dot_w, woff + j0, dots ? dots + 4 * j0 : nullptr, stats ? &sub : nullptr));
    if (stats) {
      stats->iters.insert(stats->iters.end(), sub.iters.begin(), sub.iters.end());
      stats->status.insert(stats->status.end(), sub.status.begin(), sub.status.end());
    }
  }
  return OVL_OK;
}

// Kernel low-mode deflation (Sec. 1: the smallest eigenvectors of K deflated, the rational
// covering the rest of the spectrum). With Psi the stored eigenvectors (K psi_i = lambda_i
// psi_i) and P = 1 - Psi Psi^dag,
//   sign(K) v = K [ R(K^2) P v + sum_i psi_i (psi_i, v) / |lambda_i| ],
// R the rational on the narrowed interval, so the sign's core runs on P v and the low
// modes enter y (cleaned of rounding-level components along the psi_i) before the final K
// application, whose fused epilogue stays as it is.
// kd_project: C = Psi^dag v (host, n_k x n) and *vin = P v (a P64 workspace), or v itself
// when no deflation is active (or the rational itself is differentiated).
static ovl_status kd_project(ovl_ctx* c, const Field& v, int voff, int n, const Field** vin, int* vinoff,
                             std::vector<cd>& C) {
  *vin = &v;
  *vinoff = voff;
  C.clear();
  if (c->kd_n <= 0 || c->exact_rational) return OVL_OK;
  Field* vp;
  OVL_TRY(get_field(c, "kd_vp", P64, n, &vp));
  OVL_TRY(copy_convert(c, v, voff, *vp, 0, n));
  OVL_TRY(gram_host(c, c->kd, 0, c->kd_n, *vp, 0, n, 0, C));
  std::vector<cd> m(C.size());
  for (size_t k = 0; k < C.size(); ++k) m[k] = -C[k];
  OVL_TRY(combine_host(c, c->kd, 0, c->kd_n, m, *vp, 0, n, 1));
  *vin = vp;
  *vinoff = 0;
  return OVL_OK;
}

// y <- P y + sum_i psi_i (psi_i, v) / |lambda_i| for the C of kd_project. R(K^2) P v has no
// component along the psi_i in exact arithmetic; in floating point the Krylov recurrences
// let rounding-level components along them grow (like the Lanczos polynomials outside the
// narrowed interval), so they are removed from y before the exact low-mode part is added.
static ovl_status kd_add_low(ovl_ctx* c, Field& y, int n, const std::vector<cd>& C) {
  if (C.empty()) return OVL_OK;
  const int nk = c->kd_n;
  const Field* y64 = &y;
  if (y.prec != P64 && y.prec != P32) {
    Field* t;
    OVL_TRY(get_field(c, "kd_ty", P64, n, &t));
    OVL_TRY(copy_convert(c, y, 0, *t, 0, n));
    y64 = t;
  }
  std::vector<cd> C2;
  OVL_TRY(gram_host(c, c->kd, 0, nk, *y64, 0, n, 0, C2));
  std::vector<cd> L(C.size());
  for (int i = 0; i < nk; ++i)
    for (int j = 0; j < n; ++j)
      L[(size_t)i * n + j] = C[(size_t)i * n + j] / std::fabs(c->kd_lambda[i]) - C2[(size_t)i * n + j];
  if (y.prec == P64 || y.prec == P32) return combine_host(c, c->kd, 0, nk, L, y, 0, n, 1);
  Field *t, *te;
  OVL_TRY(get_field(c, "kd_t", P64, n, &t));
  OVL_TRY(get_field(c, "kd_te", y.prec, n, &te));
  OVL_TRY(combine_host(c, c->kd, 0, nk, L, *t, 0, n, 0));
  OVL_TRY(copy_convert(c, *t, 0, *te, 0, n));
  std::vector<cd> one(n, 1.0);
  return axpby_batch(c, one, y, 0, one, *te, 0, y, 0, n);
}

// Per-system sign accuracies to the device (c->dscal), with the stopping-rule convention
// of the multi-shift CG: never past Delta (unless the rational itself is differentiated);
// positive, one error budget shared by the poles; negative, an even share per pole (the
// relaxed signs of relCG: spectrally preconditioned CGNE at mu = 0.01 lost convergence when
// its signs came close to eta_j). Returns the pointers of eta and of the (c1, c2) pairs.
static ovl_status upload_eta_coef(ovl_ctx* c, int n, const double* eta, const double* coef, double** d_eta,
                                  double** d_coef) {
  *d_eta = c->dscal;
  *d_coef = c->dscal + 4096;
  for (int j = 0; j < n; ++j) {
    double e = eta[j] > 0 ? eta[j] : c->eps_sign;
    if (e < c->delta && !c->exact_rational) e = c->delta;
    const bool shared = e < 1e-6 || c->P.solver != OVL_SOLVER_CG;
    c->hpin[j] = shared ? e : -e;
  }
  int ncopy = n;
  if (coef) {
    for (int j = 0; j < 2 * n; ++j) c->hpin[4096 + j] = coef[j];
    ncopy = 4096 + 2 * n;
  }
  OVL_CUDA(c, cudaMemcpyAsync(c->dscal, c->hpin, sizeof(double) * ncopy, cudaMemcpyHostToDevice, c->st));
  return OVL_OK;
}

// One batch of the sign function by stored-basis Lanczos (lanczos.cu): cycles of at most
// cap steps, each step the two Wilson launches (MODE_LZK, MODE_LZL) whose last block per
// system runs the scalar step, as cached CUDA graphs of kGraphIters steps without profiling;
// then the per-pole tridiagonal solves, one pass over the stored basis, and the final
// Wilson application with the overlap / sign epilogue.
static ovl_status sign_op_batch_lz(ovl_ctx* c, int mode, const Field& v, int voff, Field& out, int ooff, int n,
                                   const double* eta, double c1, double c2, const double* coef, int herm,
                                   const Field* dot_w, int woff, double* dots, SignStats* stats, int cap) {
  const int PL = mode == SIGN64 ? P64 : mode == SIGN32 ? P32 : mode == SIGN16 ? P16 : P64E;
  const int PR = mode == SIGN64 ? P64 : mode == SIGN64E ? P64E : P32;   // y
  const int PB = PL;                                                      // basis and t
  const int V = c->V;
  const std::string tag = std::to_string(mode);
  Field Wv;
  Field* W = &Wv;
  Field *t, *y;
  OVL_TRY(lz_pool_field(c, PB, cap * n, &Wv));
  struct PoolBusy {
    ovl_ctx* c;
    ~PoolBusy() { c->lz_pool_busy = false; }
  } busy{c};
  c->lz_pool_busy = true;
  OVL_TRY(get_field(c, "lz_t" + tag, PB, n, &t));
  OVL_TRY(get_field(c, "lz_y" + tag, PR, n, &y));
  OVL_TRY(ensure_partials(c, n));
  OVL_TRY(ensure_lz(c, n, cap));
  const Shape sh = make_shape(V, n);
  double *d_eta, *d_coef;
  OVL_TRY(upload_eta_coef(c, n, eta, coef, &d_eta, &d_coef));
  const LinkRef L = links_of(c, PL);
  const int wcls = PL == P64E ? 8 : PL;
  const double lbytes = (PL == P64E ? 576.0 : PL == P64 ? 384.0 : PL == P32 ? 192.0 : 96.0) * V;
  const double sbytes = (double)spinor_bytes(PB) * V, rbytes = (double)spinor_bytes(PR) * V;
  double* ahist = c->lz_hist;
  double* bhist = c->lz_hist + (size_t)c->lz_n * c->lz_cap;
  const int hcap = c->lz_cap;   // row length of the histories and coefficient buffers
  const LzCtl ctl{c->lz, c->lz_ctr, ahist, bhist, hcap, c->dpoles};
  ProfPair pp;

  const Field* vin;
  int vinoff;
  std::vector<cd> kdC;
  OVL_TRY(kd_project(c, v, voff, n, &vin, &vinoff, kdC));
  prof_begin(c, 4, &pp);
  launch_lz_init(vin->prec, PB, PR, vin->ref(vinoff), W->ref(), y->ref(), n, V, c->partials, c->st);
  prof_end(c, &pp, (double)n * V * (spinor_bytes(vin->prec) + spinor_bytes(PB) + spinor_bytes(PR)));
  prof_begin(c, 5, &pp);
  launch_lz_start(c->lz, c->partials, sh.nsb, n, c->dpoles, d_eta, c->P.mscg_max, cap, 1, c->st);
  prof_end(c, &pp, 0.0);
  OVL_TRY(check_launch(c, __func__));

  cudaGraphExec_t gexec = nullptr;
  if (!c->prof.on && c->P.use_graphs) {
    const std::vector<unsigned long long> key = {
        1000ull + (unsigned long long)PB, (unsigned long long)PL, (unsigned long long)n, (unsigned long long)hcap,
        (unsigned long long)(uintptr_t)W->data, (unsigned long long)(uintptr_t)t->data,
        // FP16 storage: the per-site scales of the pooled basis sit after its data, at an
        // offset that depends on the cycle length, so they are part of the key
        (unsigned long long)(uintptr_t)W->norm, (unsigned long long)(uintptr_t)t->norm,
        (unsigned long long)(uintptr_t)c->partials, (unsigned long long)(uintptr_t)c->lz,
        (unsigned long long)(uintptr_t)c->lz_hist, (unsigned long long)(uintptr_t)L.data,
        (unsigned long long)L.variant};
    OVL_TRY(ms_graph(c, key, &gexec, [&](cudaStream_t cs) {
      for (int k = 0; k < kGraphIters; ++k) {
        launch_wilson_lzK(PB, PL, PB, c->g, c->kappa, L, W->ref(), t->ref(), n, c->partials, ctl, cs);
        launch_wilson_lzL(PB, PL, PB, c->g, c->kappa, L, t->ref(), W->ref(), n, c->partials, ctl, cs);
      }
    }));
  }
  int* hflags = reinterpret_cast<int*>(c->hpin + 8192);
  int total = 0;
  long long live = 0, wreads = 0;
  int itmax = 0;
  double comb_bytes = 0.0;
  std::vector<int> it(n, 0), stt(n, 0);
  for (int cycle = 0;; ++cycle) {
    int chunk = 8;
    while (true) {
      if (gexec) {
        for (int k = 0; k < chunk; k += kGraphIters) OVL_CUDA(c, cudaGraphLaunch(gexec, c->st));
      } else {
        for (int k = 0; k < chunk; ++k) {
          prof_begin(c, wcls, &pp);
          launch_wilson_lzK(PB, PL, PB, c->g, c->kappa, L, W->ref(), t->ref(), n, c->partials, ctl, c->st);
          prof_end(c, &pp, 0.0);
          prof_begin(c, wcls, &pp);
          launch_wilson_lzL(PB, PL, PB, c->g, c->kappa, L, t->ref(), W->ref(), n, c->partials, ctl, c->st);
          prof_end(c, &pp, 0.0);
        }
      }
      total += chunk;
      OVL_TRY(check_launch(c, __func__));
      OVL_CUDA(c, cudaMemcpy2DAsync(hflags, sizeof(int), &c->lz[0].done, sizeof(LzRhs), sizeof(int), n,
                                    cudaMemcpyDeviceToHost, c->st));
      OVL_CUDA(c, cudaStreamSynchronize(c->st));
      bool all = true;
      for (int j = 0; j < n; ++j) all = all && hflags[j];
      if (all) break;
      if (total > c->P.mscg_max + 16 * (cycle + 1)) break;
      chunk = std::min(32, chunk * 2);
    }
    // this cycle's part of y
    prof_begin(c, 5, &pp);
    launch_lz_coef(c->lz, ahist, bhist, hcap, c->dpoles, c->lz_Y, c->lz_coefW, n, c->st);
    prof_end(c, &pp, 0.0);
    // steps of this cycle per system (the basis vectors the combine reads)
    OVL_CUDA(c, cudaMemcpy2DAsync(hflags, sizeof(int), &c->lz[0].j, sizeof(LzRhs), sizeof(int), n,
                                  cudaMemcpyDeviceToHost, c->st));
    OVL_CUDA(c, cudaStreamSynchronize(c->st));
    long long kk = 0;
    for (int j = 0; j < n; ++j) kk += hflags[j];
    const double cb = (double)kk * sbytes + (double)n * 2.0 * rbytes;
    comb_bytes += cb;
    prof_begin(c, 3, &pp);
    launch_lz_combine(PB, PR, W->ref(), y->ref(), c->lz_coefW, c->lz, hcap, n, V, c->st);
    prof_end(c, &pp, cb);
    OVL_TRY(check_launch(c, __func__));
    // cycles that filled up continue from their last basis vector
    OVL_CUDA(c, cudaMemcpy2DAsync(hflags, sizeof(int), &c->lz[0].status, sizeof(LzRhs), sizeof(int), n,
                                  cudaMemcpyDeviceToHost, c->st));
    OVL_CUDA(c, cudaMemcpy2DAsync(hflags + 4096, sizeof(int), &c->lz[0].finished, sizeof(LzRhs), sizeof(int), n,
                                  cudaMemcpyDeviceToHost, c->st));
    OVL_CUDA(c, cudaStreamSynchronize(c->st));
    bool more = false;
    for (int j = 0; j < n; ++j) more = more || (hflags[j] == 3 && !hflags[4096 + j]);
    if (!more) break;
    prof_begin(c, 4, &pp);
    launch_lz_restart(PB, W->ref(), c->lz, n, V, c->partials, c->st);
    prof_end(c, &pp, 2.0 * n * sbytes);
    launch_lz_start(c->lz, c->partials, sh.nsb, n, c->dpoles, d_eta, c->P.mscg_max, cap, 0, c->st);
    OVL_TRY(check_launch(c, __func__));
  }
  OVL_TRY(kd_add_low(c, *y, n, kdC));
  // final Wilson application with the overlap / sign epilogue
  double* d_part = dot_w ? c->partials : nullptr;
  prof_begin(c, wcls, &pp);
  launch_wilson_ovl(PR, PL, out.prec, c->g, c->kappa, L, y->ref(), v.ref(voff), out.ref(ooff),
                    dot_w ? dot_w->ref(woff) : SpinorRef{nullptr, nullptr, V}, n, c1, c2, coef ? d_coef : nullptr,
                    herm, d_part, c->st);
  prof_end(c, &pp, (double)n * V * (spinor_bytes(PR) + 2.0 * spinor_bytes(out.prec)) + lbytes);
  OVL_TRY(check_launch(c, __func__));
  if (dot_w) OVL_TRY(reduce_to_host_nv(c, sh.nsb, n, dots, 4));
  long long* hll = reinterpret_cast<long long*>(c->hpin + 12288);
  OVL_CUDA(c, cudaMemcpy2DAsync(hflags, sizeof(int), &c->lz[0].total, sizeof(LzRhs), sizeof(int), n,
                                cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaMemcpy2DAsync(hflags + 4096, sizeof(int), &c->lz[0].status, sizeof(LzRhs), sizeof(int), n,
                                cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaMemcpy2DAsync(hll, sizeof(long long), &c->lz[0].w_reads, sizeof(LzRhs), sizeof(long long), n,
                                cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  for (int j = 0; j < n; ++j) {
    it[j] = hflags[j];
    stt[j] = hflags[4096 + j];
    live += it[j];
    wreads += hll[j];
    itmax = std::max(itmax, it[j]);
  }
  c->wcalls[PL] += 2 * live + n;
  double emin = 1e300;
  for (int j = 0; j < n; ++j) emin = std::min(emin, eta[j] > 0 ? eta[j] : c->eps_sign);
  if (!c->exact_rational) emin = std::max(emin, c->delta);
  int& km = c->lz_kmax[mode][eta_decade(emin)];
  km = std::max(km, itmax);
  if (c->prof.on) {
    // algorithmic bytes: the K mode reads W_j and writes t, the L mode reads t and W_j
    // (and W_{j-1} after the first step) and writes W_{j+1}; links once per launch
    c->prof.bytes[wcls] += (double)live * 4.0 * sbytes + (double)wreads * sbytes + 2.0 * lbytes * itmax;
    c->prof.units[wcls] += (2.0 * (double)live + n) * V;
    c->prof.units[3] += comb_bytes / std::max(1.0, sbytes) * V;
  }
  if (stats) {
    stats->iters = it;
    stats->status = stt;
  }
  for (int j = 0; j < n; ++j) {
    if (stt[j] == 2) {
      char m[160];
      snprintf(m, sizeof(m), "Lanczos breakdown in the sign function (system %d, step %d)", j, it[j]);
      return set_err(c, OVL_EBREAKDOWN, m);
    }
  }
  for (int j = 0; j < n; ++j) {
    if (stt[j] == 1) {
      char m[200];
      snprintf(m, sizeof(m),
               "Lanczos sign stopped at the iteration limit (mscg_max = %d) before the sign accuracy %.3e was met "
               "(system %d, %d steps)",
               c->P.mscg_max, eta[j], j, it[j]);
      return set_err(c, OVL_ENOCONV, m);
    }
  }
  return OVL_OK;
}

static ovl_status sign_op_batch(ovl_ctx* c, int mode, const Field& v, int voff, Field& out, int ooff, int n,
                                const double* eta, double c1, double c2, const double* coef, int herm,
                                const Field* dot_w, int woff, double* dots, SignStats* stats) {
  const int PL = mode == SIGN64 ? P64 : mode == SIGN32 ? P32 : mode == SIGN16 ? P16 : P64E;
  const int PR = mode == SIGN64 ? P64 : mode == SIGN64E ? P64E : P32;
  const int PP = PL;
  const int V = c->V;
  const int np = c->npoles;
  const std::string tag = std::to_string(mode);
  Field *r, *y, *t, *pb;
  OVL_TRY(get_field(c, "ms_r" + tag, PR, n, &r));
  OVL_TRY(get_field(c, "ms_y" + tag, PR, n, &y));
  OVL_TRY(get_field(c, "ms_t" + tag, PP, n, &t));
  OVL_TRY(get_field(c, "ms_p" + tag, PP, np * n, &pb));
  OVL_TRY(ensure_partials(c, n));
  OVL_TRY(ensure_ms(c, n));
  const Shape sh = make_shape(V, n);
  // per-system eta and (c1, c2) to the device
  double *d_eta, *d_coef;
  OVL_TRY(upload_eta_coef(c, n, eta, coef, &d_eta, &d_coef));
  const LinkRef L = links_of(c, PL);
  const int wcls = PL == P64E ? 8 : PL;  // profiler class of the Wilson launches
  // algorithmic link bytes per site and launch: four 18-real FP64 links for the
  // double-float kernel (its eight-slot field stores each link twice, forward and
  // transposed, which is a layout choice, not work), four 12-real links otherwise
  const double lbytes = (PL == P64E ? 576.0 : PL == P64 ? 384.0 : PL == P32 ? 192.0 : 96.0) * V;
  const double sbytes = (double)spinor_bytes(PP) * V, rbytes = (double)spinor_bytes(PR) * V;
  ProfPair pp;

  const Field* vin;
  int vinoff;
  std::vector<cd> kdC;
  OVL_TRY(kd_project(c, v, voff, n, &vin, &vinoff, kdC));
  prof_begin(c, 4, &pp);
  launch_ms_init(vin->prec, PR, PP, vin->ref(vinoff), r->ref(), pb->ref(), y->ref(), np, n, V, c->partials, c->st);
  prof_end(c, &pp, (double)n * V * (spinor_bytes(vin->prec) + 2 * spinor_bytes(PR) + np * spinor_bytes(PP)));
  prof_begin(c, 5, &pp);
  launch_ms_scalar0(c->ms, c->partials, sh.nsb, n, c->dpoles, d_eta, c->P.mscg_max, c->st);
  prof_end(c, &pp, 0.0);
  OVL_TRY(check_launch(c, __func__));

  int* hdone = reinterpret_cast<int*>(c->hpin + 8192);
  int total = 0;
  int chunk = 8;
  // Without profiling, the iterations run as a CUDA graph of kGraphIters iterations,
  // captured once per field configuration and replayed: one graph launch instead of
  // 5 kGraphIters kernel launches (a single-system step on 16^3 x 32 is ~50 us of
  // kernels, comparable to the launch overhead of its 5 launches).
  cudaGraphExec_t gexec = nullptr;
  if (!c->prof.on && c->P.use_graphs) {
    const std::vector<unsigned long long> key = {
        (unsigned long long)PP, (unsigned long long)PL, (unsigned long long)PR, (unsigned long long)n,
        (unsigned long long)np, (unsigned long long)(uintptr_t)pb->data, (unsigned long long)(uintptr_t)t->data,
        (unsigned long long)(uintptr_t)r->data, (unsigned long long)(uintptr_t)y->data,
        (unsigned long long)(uintptr_t)pb->norm, (unsigned long long)(uintptr_t)t->norm,
        (unsigned long long)(uintptr_t)r->norm, (unsigned long long)(uintptr_t)y->norm,
        (unsigned long long)(uintptr_t)c->partials, (unsigned long long)(uintptr_t)c->ms,
        (unsigned long long)(uintptr_t)L.data, (unsigned long long)L.variant};
    OVL_TRY(ms_graph(c, key, &gexec, [&](cudaStream_t cs) {
      for (int k = 0; k < kGraphIters; ++k) {
        launch_wilson_K(PP, PL, PP, c->g, c->kappa, L, pb->ref(), t->ref(), n, c->partials, c->ms, cs);
        launch_ms_scalar1(c->ms, c->partials, sh.nsb, n, c->dpoles, cs);
        launch_wilson_mscg_r(PP, PL, PR, PP, c->g, c->kappa, L, t->ref(), pb->ref(), r->ref(), n,
                             c->hpoles.sigma0, c->partials, c->ms, cs);
        launch_ms_scalar2(c->ms, c->partials, sh.nsb, n, c->dpoles, cs);
        launch_ms_update(PR, PP, r->ref(), pb->ref(), y->ref(), np, n, V, c->ms, cs);
      }
    }));
  }
  while (true) {
    if (gexec) {
      for (int k = 0; k < chunk; k += kGraphIters) OVL_CUDA(c, cudaGraphLaunch(gexec, c->st));
    } else for (int k = 0; k < chunk; ++k) {
      prof_begin(c, wcls, &pp);
      launch_wilson_K(PP, PL, PP, c->g, c->kappa, L, pb->ref(), t->ref(), n, c->partials, c->ms, c->st);
      prof_end(c, &pp, 0.0);
      prof_begin(c, 5, &pp);
      launch_ms_scalar1(c->ms, c->partials, sh.nsb, n, c->dpoles, c->st);
      prof_end(c, &pp, 0.0);
      prof_begin(c, wcls, &pp);
      launch_wilson_mscg_r(PP, PL, PR, PP, c->g, c->kappa, L, t->ref(), pb->ref(), r->ref(), n, c->hpoles.sigma0,
                           c->partials, c->ms, c->st);
      prof_end(c, &pp, 0.0);
      prof_begin(c, 5, &pp);
      launch_ms_scalar2(c->ms, c->partials, sh.nsb, n, c->dpoles, c->st);
      prof_end(c, &pp, 0.0);
      prof_begin(c, 3, &pp);
      launch_ms_update(PR, PP, r->ref(), pb->ref(), y->ref(), np, n, V, c->ms, c->st);
      prof_end(c, &pp, 0.0);
    }
    total += chunk;
    OVL_TRY(check_launch(c, __func__));
    OVL_CUDA(c, cudaMemcpy2DAsync(hdone, sizeof(int), &c->ms[0].done, sizeof(MsRhs), sizeof(int), n,
                                  cudaMemcpyDeviceToHost, c->st));
    OVL_CUDA(c, cudaStreamSynchronize(c->st));
    bool all = true;
    for (int j = 0; j < n; ++j) all = all && hdone[j];
    if (all) break;
    if (total > c->P.mscg_max + 16) break;
    chunk = std::min(32, chunk * 2);
  }
  OVL_TRY(kd_add_low(c, *y, n, kdC));
  // final Wilson application with the overlap / sign epilogue
  double* d_part = dot_w ? c->partials : nullptr;
  prof_begin(c, wcls, &pp);
  launch_wilson_ovl(PR, PL, out.prec, c->g, c->kappa, L, y->ref(), v.ref(voff), out.ref(ooff),
                    dot_w ? dot_w->ref(woff) : SpinorRef{nullptr, nullptr, V}, n, c1, c2, coef ? d_coef : nullptr,
                    herm, d_part, c->st);
  prof_end(c, &pp, (double)n * V * (spinor_bytes(PR) + 2.0 * spinor_bytes(out.prec)) + lbytes);
  OVL_TRY(check_launch(c, __func__));
  if (dot_w) OVL_TRY(reduce_to_host_nv(c, sh.nsb, n, dots, 4));
  // iteration counts, status and byte counters
  std::vector<int> it(n), stt(n);
  std::vector<long long> prd(n), pwr(n);
  OVL_CUDA(c, cudaMemcpy2DAsync(hdone, sizeof(int), &c->ms[0].iter, sizeof(MsRhs), sizeof(int), n,
                                cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaMemcpy2DAsync(hdone + 4096, sizeof(int), &c->ms[0].status, sizeof(MsRhs), sizeof(int), n,
                                cudaMemcpyDeviceToHost, c->st));
  long long* hll = reinterpret_cast<long long*>(c->hpin + 12288);
  OVL_CUDA(c, cudaMemcpy2DAsync(hll, sizeof(long long), &c->ms[0].p_reads, sizeof(MsRhs), sizeof(long long), n,
                                cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaMemcpy2DAsync(hll + 4096, sizeof(long long), &c->ms[0].p_writes, sizeof(MsRhs), sizeof(long long),
                                n, cudaMemcpyDeviceToHost, c->st));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  long long live = 0, pr = 0, pw = 0;
  int itmax = 0;
  for (int j = 0; j < n; ++j) {
    it[j] = hdone[j];
    stt[j] = hdone[4096 + j];
    live += it[j];
    itmax = std::max(itmax, it[j]);
    pr += hll[j];
    pw += hll[4096 + j];
  }
  c->wcalls[PL] += 2 * live + n;
  if (c->prof.on) {
    // algorithmic bytes of the chunked launches from the device-side live counts:
    // MODE_K reads p_0 and writes t, MODE_R reads t, p_0, r and writes r, the links
    // are read once per launch; the update reads r, y, the pole vectors and writes
    // y and the still-active pole vectors.
    c->prof.bytes[wcls] += (double)live * (4.0 * sbytes + 2.0 * rbytes) + 2.0 * lbytes * itmax;
    c->prof.bytes[3] += (double)live * 3.0 * rbytes + (double)(pr + pw) * sbytes;
    // work units: site applications of the Wilson kernel, site passes of the update
    c->prof.units[wcls] += (2.0 * (double)live + n) * V;
    c->prof.units[3] += (double)live * V;
  }
  if (stats) {
    stats->iters = it;
    stats->status = stt;
  }
  for (int j = 0; j < n; ++j) {
    if (stt[j] == 2) {
      char m[160];
      snprintf(m, sizeof(m), "multi-shift CG breakdown in the sign function (system %d, iteration %d)", j, it[j]);
      return set_err(c, OVL_EBREAKDOWN, m);
    }
  }
  // a system that reached the iteration limit has a sign less accurate than asked for
  // (the pole stopping rule of Sec. 3 was not met): the caller has to know
  for (int j = 0; j < n; ++j) {
    if (stt[j] == 1) {
      char m[200];
      snprintf(m, sizeof(m),
               "multi-shift CG stopped at the iteration limit (mscg_max = %d) before the sign accuracy "
               "%.3e was met (system %d, %d iterations)",
               c->P.mscg_max, eta[j], j, it[j]);
      return set_err(c, OVL_ENOCONV, m);
    }
  }
  return OVL_OK;
}

}  // namespace ovl
