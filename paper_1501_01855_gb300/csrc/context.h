// Library-internal state of one overlap context: gauge field in every storage
// precision, Zolotarev poles, device workspaces, profiling, error text.
#pragma once
#include <cuda_runtime.h>

#include <complex>
#include <map>
#include <string>
#include <vector>

#include "../../include/overlap.h"
#include "kernels.h"

namespace ovl {

using cd = std::complex<double>;

struct ProfPair {
  cudaEvent_t a, b;
  int cls;
  double bytes;
};

struct Profiler {
  bool on = false;
  long long launches[OVL_PROF_CLASSES] = {0};
  double ms[OVL_PROF_CLASSES] = {0};
  double bytes[OVL_PROF_CLASSES] = {0};
  double units[OVL_PROF_CLASSES] = {0};
  std::vector<ProfPair> pending;
  std::vector<cudaEvent_t> pool;
};

// Sign-function precision modes (Sec. 3: single precision when the required
// accuracy allows; FP16 storage extends the same idea one step further).
// SIGN64E: FP64-accurate sign computed in double-float on the FP32 pipes.
enum SignMode { SIGN64 = 0, SIGN32 = 1, SIGN16 = 2, SIGN64E = 3 };

// An instantiated CUDA graph of G multi-shift CG iterations (5 launches each), keyed by
// everything its launches capture (field pointers, precisions, counts, constants).
struct MsGraph {
  std::vector<unsigned long long> key;
  cudaGraphExec_t exec = nullptr;
  long long last_use = 0;
};

struct SignStats {
  std::vector<int> iters;     // multi-shift CG iterations per system
  std::vector<int> status;    // 0 converged, 1 iteration limit, 2 breakdown
};

struct ovl_ctx_impl;
}  // namespace ovl

struct ovl_ctx {
  ovl::Geom g;
  int V = 0;
  double m0 = 0, kappa = 0, mu = 0;
  int npoles = 0;
  double eps_sign = 0, delta = 0, za = 0, zb = 0;
  std::vector<double> omega, sigma;
  ovl_params P;
  cudaStream_t st = nullptr;
  int device = 0;
  void* link[4] = {nullptr, nullptr, nullptr, nullptr};  // P64, P32, P16, P64E 12-real layouts
  int wvar[4] = {0, 0, 0, 0};                            // Wilson-kernel variant per precision
  float wtime[4][4] = {{0}};                             // autotuner timings (ms per launch)
  int wvar_multi[4] = {0, 0, 0, 0};                      // the same for launches of >= 4 systems
  float wtime_multi[4][4] = {{0}};
  ovl::Poles hpoles;
  ovl::Poles* dpoles = nullptr;
  std::map<std::string, ovl::Field> ws;
  double* partials = nullptr;
  size_t partials_n = 0;
  double* dred = nullptr;        // reduced per-rhs pairs (device), 2 * 4096
  double* dscal = nullptr;       // per-rhs scalars (device), 64 * 4096
  int* dint = nullptr;           // per-rhs ints (device), 4096
  ovl::MsRhs* ms = nullptr;
  int ms_n = 0;
  ovl::LzRhs* lz = nullptr;      // stored-basis Lanczos state per system
  int lz_n = 0;
  double* lz_hist = nullptr;     // alpha_j and beta_j histories, 2 * lz_n * lz_cap doubles
  double* lz_Y = nullptr;        // per-pole tridiagonal solves, lz_n * npoles * 2 lz_cap doubles
  double* lz_coefW = nullptr;    // coefficients of the stored vectors, lz_n * lz_cap doubles
  unsigned int* lz_ctr = nullptr;  // arrival counters of the fused scalar steps, lz_n
  int lz_cap = 0;
  void* lz_pool = nullptr;       // stored Lanczos bases of every sign precision (one at a time)
  size_t lz_pool_bytes = 0;
  bool lz_pool_busy = false;     // a sign application holds a view of the pool
  int lz_kmax[4][17] = {{0}};    // most Lanczos steps seen per sign mode and decade of eta
  double* hpin = nullptr;        // pinned host staging for scalars, 64 * 4096 doubles
  void* hstage = nullptr;        // pinned host staging for spinor copies
  size_t hstage_bytes = 0;
  double* dwork = nullptr;       // Gram work buffer
  size_t dwork_n = 0;
  size_t ring_pos = 0;           // scalar upload ring in hpin / dscal, [32768, 262144)
  cudaEvent_t stage_ev = nullptr;  // last copy out of hstage
  cudaStream_t cap_st = nullptr;   // private stream for graph capture (the context stream may be the legacy one)
  std::vector<ovl::MsGraph> graphs;  // cached multi-shift CG iteration graphs
  long long graph_clock = 0;
  bool exact_rational = false;   // solve shifted systems past Delta (gradient of the rational)
  // kernel low-mode deflation of the sign function (Sec. 1): eigenvectors of K with the
  // smallest |lambda| (FP64), their eigenvalues, and the interval and pole count the rational
  // had before it was narrowed to the rest of the spectrum
  ovl::Field kd;
  int kd_n = 0;
  std::vector<double> kd_lambda;
  double za0 = 0.0;
  int npoles0 = 0;
  std::string err;
  ovl::Profiler prof;
  long long wcalls[4] = {0, 0, 0, 0};  // Wilson applications by precision
};

struct ovl_defl {
  ovl_ctx* ctx = nullptr;
  int n = 0;            // vectors held
  int cap = 0;          // capacity of v, w
  ovl::Field v;         // approximate low eigenvectors psi_i of D^dag D (and of gamma5 D)
  ovl::Field w;         // w_i = gamma5 eps(K) psi_i, so that D(mu) psi_i = (1+mu)/2 psi_i + (1-mu)/2 w_i
  std::vector<double> ritz, res;
  double mu = 0;        // mass at which the Ritz values were computed
  bool per_vector = false;   // Sec. 4 per-vector alpha_j instead of the least-squares solve
  bool prepared = false;
  std::vector<std::complex<double>> VV, WW, WV, G5VV, G5VW;   // Gram blocks over psi and w
};

namespace ovl {

// error helpers
ovl_status set_err(ovl_ctx* c, ovl_status s, const std::string& m);
ovl_status cuda_check(ovl_ctx* c, cudaError_t e, const char* what);
#define OVL_CUDA(c, call)                                     \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ovl::cuda_check(c, _e, #call); \
  } while (0)
#define OVL_TRY(expr)                  \
  do {                                 \
    ovl_status _s = (expr);            \
    if (_s != OVL_OK) return _s;       \
  } while (0)

// cudaGetLastError plus the unsupported-precision flag of the launchers
ovl_status check_launch(ovl_ctx* c, const char* where);

// workspace
ovl_status get_field(ovl_ctx* c, const std::string& name, int prec, int n, Field** out);
void free_field(Field& f);
ovl_status ensure_partials(ovl_ctx* c, int nrhs);
ovl_status ensure_ms(ovl_ctx* c, int nrhs);
ovl_status ensure_lz(ovl_ctx* c, int nrhs, int cap);
// a view of n fields of precision prec over the context's basis pool (grown on demand; the
// view is not owned and must not be passed to free_field)
ovl_status lz_pool_field(ovl_ctx* c, int prec, int n, Field* out);
// free every cached workspace, graph and pool of the context (what the next call needs is
// allocated again)
void trim_workspaces(ovl_ctx* c);
ovl_status ensure_stage(ovl_ctx* c, size_t bytes);
ovl_status ensure_work(ovl_ctx* c, size_t ndoubles);

// profiling
void prof_begin(ovl_ctx* c, int cls, ProfPair* p);
void prof_end(ovl_ctx* c, ProfPair* p, double bytes);
void prof_flush(ovl_ctx* c);

LinkRef links_of(const ovl_ctx* c, int prec);

// reductions: partials -> host pairs (synchronises the stream)
ovl_status reduce_to_host(ovl_ctx* c, int nsb, int nrhs, double* host_pairs);
// the first nv of the NVRED partial sums per system
ovl_status reduce_to_host_nv(ovl_ctx* c, int nsb, int nrhs, double* out, int nv);

// I/O between caller buffers and internal fields
ovl_status import_spinors(ovl_ctx* c, const void* src, int dtype, int on_device, int n, Field& dst, int off);
ovl_status export_spinors(ovl_ctx* c, void* dst, int dtype, int on_device, int n, const Field& src, int off);

// sign function: out = c1 v + c2 gamma5 K y (times gamma5 if herm), y = sum_i omega_i (K^2+sigma_i)^-1 v,
// every system stopped at its own relative accuracy eta[j]. dot_w (may be null) requests
// {Re (w_j, out_j), Im (w_j, out_j), ||out_j||^2, ||w_j||^2} into dots (host, 4n). coef (host,
// may be null) gives per-system (c1, c2).
ovl_status sign_op(ovl_ctx* c, int mode, const Field& v, int voff, Field& out, int ooff, int n, const double* eta,
                   double c1, double c2, const double* coef, int herm, const Field* dot_w, int woff, double* dots,
                   SignStats* stats);
int choose_mode(const ovl_ctx* c, double eta);

// Zolotarev rational with n_poles poles on [a, b] (ascending sigma), its error bound and the
// per-pole bounds, to the context and the device; OVL_EAPPROX when Delta exceeds eps_sign.
ovl_status set_poles(ovl_ctx* c, int n_poles, double a, double b);
// Extreme eigenvalues of K^2 by `steps` Lanczos steps from a fixed random vector; with nproj
// > 0 on the complement of the first nproj (orthonormal) vectors of *proj.
ovl_status lanczos_bounds(ovl_ctx* c, int steps, double* lmin, double* lmax, const Field* proj = nullptr,
                          int nproj = 0);

// Upload count doubles of per-system scalars through the pinned ring; returns the
// device copy (valid for kernels issued later on the context stream).
ovl_status upload(ovl_ctx* c, const double* host, int count, const double** dev);

// gamma5 K applied to n systems in FP64 etc. lives in the solvers; this is the plain Wilson kernel
ovl_status wilson_apply_field(ovl_ctx* c, int prec, const Field& in, int ioff, Field& out, int ooff, int n);
}  // namespace ovl
