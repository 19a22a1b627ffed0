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

ovl_status ensure_stage(ovl_ctx* c, size_t bytes) {
  if (bytes <= c->hstage_bytes) return OVL_OK;
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

// Systems per multi-shift solve are capped so that the pole vectors of one batch stay
// within kPoleBytes (24 poles x 36 systems of 24^3 x 48 in double-float would be 110 GB);
// larger requests run as consecutive sub-batches.
static constexpr double kPoleBytes = 64e9;
ovl_status sign_op(ovl_ctx* c, int mode, const Field& v, int voff, Field& out, int ooff, int n, const double* eta,
                   double c1, double c2, const double* coef, int herm, const Field* dot_w, int woff, double* dots,
                   SignStats* stats) {
  if (n <= 0) return OVL_OK;
  const int PP = mode == SIGN64 ? P64 : mode == SIGN32 ? P32 : mode == SIGN16 ? P16 : P64E;
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
  double* d_eta = c->dscal;
  double* d_coef = c->dscal + 4096;
  for (int j = 0; j < n; ++j) {
    double e = eta[j] > 0 ? eta[j] : c->eps_sign;
    // the sign is never more accurate than Delta, so no pole is solved past it, except
    // when the rational itself is being differentiated (gauge-link gradient)
    if (e < c->delta && !c->exact_rational) e = c->delta;
    // stopping rule (see ms_scalar2): one error budget shared by the poles, except for the
    // relaxed signs of relCG (spectrally preconditioned CGNE lost convergence at mu = 0.01
    // when its signs came close to eta_j), which keep an even share per pole (negative)
    const bool shared = e < 1e-6 || c->P.solver != OVL_SOLVER_CG;
    c->hpin[j] = shared ? e : -e;
  }
  int ncopy = n;
  if (coef) {
    for (int j = 0; j < 2 * n; ++j) c->hpin[4096 + j] = coef[j];
    ncopy = 4096 + 2 * n;
  }
  OVL_CUDA(c, cudaMemcpyAsync(c->dscal, c->hpin, sizeof(double) * ncopy, cudaMemcpyHostToDevice, c->st));
  const LinkRef L = links_of(c, PL);
  const int wcls = PL == P64E ? 8 : PL;  // profiler class of the Wilson launches
  // algorithmic link bytes per site and launch: four 18-real FP64 links for the
  // double-float kernel (its eight-slot field stores each link twice, forward and
  // transposed, which is a layout choice, not work), four 12-real links otherwise
  const double lbytes = (PL == P64E ? 576.0 : PL == P64 ? 384.0 : PL == P32 ? 192.0 : 96.0) * V;
  const double sbytes = (double)spinor_bytes(PP) * V, rbytes = (double)spinor_bytes(PR) * V;
  ProfPair pp;

  prof_begin(c, 4, &pp);
  launch_ms_init(v.prec, PR, PP, v.ref(voff), r->ref(), pb->ref(), y->ref(), np, n, V, c->partials, c->st);
  prof_end(c, &pp, (double)n * V * (spinor_bytes(v.prec) + 2 * spinor_bytes(PR) + np * spinor_bytes(PP)));
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
