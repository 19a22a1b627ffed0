// Host-side launch interface of the liboverlap kernels. Every launcher issues
// its work on the given stream and returns immediately; none synchronises.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdio.h>

#include "common.cuh"

namespace ovl {

// A launcher asked for a precision combination that has no instantiation records
// it here (nothing is launched); the host code turns it into OVL_EINVAL.
void note_bad_combo(const char* where);
bool take_bad_combo();

constexpr int NPMAX = 64;       // maximum Zolotarev poles
constexpr int BX = 64;          // sites per block (x dimension of every site kernel)
constexpr int NVRED = 4;        // doubles per (rhs, block) reduction partial

// A batch of spinor fields owned by the library.
struct Field {
  int prec = -1;
  int n = 0;
  int V = 0;
  void* data = nullptr;
  float* norm = nullptr;
  size_t chunk_bytes() const { return (size_t)n * V * spinor_site_bytes(prec); }
  SpinorRef ref(int off = 0) const {
    SpinorRef r;
    const size_t per = (size_t)V * spinor_site_bytes(prec);
    r.data = data ? (void*)((char*)data + per * off) : nullptr;
    r.norm = norm ? norm + (size_t)V * off : nullptr;
    r.V = V;
    return r;
  }
};

// Per-system multi-shift CG state, device resident (Sec. 3: the shifted systems
// (K^2 + sigma_i) x_i = v of the Zolotarev sum solved with one Krylov space).
struct MsRhs {
  double rr, alpha, alpha_prev, beta_prev, thr;
  double consumed;   // error bound frozen by the poles already dropped
  int active, nact_y, done, iter, status, maxit;
  long long p_reads, p_writes;   // pole-vector passes of the fused update (bytes accounting)
  double zeta[NPMAX], zeta_prev[NPMAX], zeta_next[NPMAX];
  double coef_y[NPMAX], coef_r[NPMAX], coef_p[NPMAX], coef_a[NPMAX];
};

// Per-system state of the stored-basis Lanczos evaluation of the Zolotarev sum (Sec. 3),
// device resident. The Krylov basis of K^2 is kept in HBM (unnormalised vectors W_l,
// v_l = W_l / n_l), so that every pole's Galerkin solution comes from its own small
// tridiagonal solve and one combination of the stored vectors, with no per-pole vector
// traffic. One cycle holds at most `cap` basis vectors; a cycle that fills up restarts
// from the last vector, to which every pole's residual is parallel.
struct LzRhs {
  double vnorm;        // n_0 = ||W_0|| of this cycle
  double inv_n;        // 1 / n_j: K-mode scale of the current basis vector
  double inv_nprev;    // 1 / n_{j-1}
  double a, b;         // L-mode coefficients alpha_j / n_j and beta_{j-1} / n_{j-1}
  double alpha;        // alpha_j = (v_j, K^2 v_j)
  double beta_prev;    // beta_{j-1}
  double thr;          // error budget eta ||v|| of the caller's vector
  double err;          // current error bound sum_i |w_i| g_i rho_i
  int j;               // basis vectors completed in this cycle (next K-mode input W_j)
  int done;            // 1: this cycle has stopped
  int status;          // 0 converged, 1 iteration limit, 2 breakdown, 3 cycle full (restart)
  int total;           // iterations over all cycles
  int maxit, cap;      // iteration limit, basis slots per cycle
  int finished;        // 1: no more cycles for this system
  int cycles;
  int even;            // 1: stop when every pole is within thr / N_Z (relaxed signs of relCG)
  long long w_reads;   // basis vector passes of the L mode (bytes accounting)
  double w[NPMAX];     // pole weights of this cycle (omega_i in the first)
  double d[NPMAX];     // LDL^T pivots of T_j + sigma_i
  double rho[NPMAX];   // residual norms of the shifted Galerkin solutions
};

// Pole data of one context, device resident.
struct Poles {
  int n;
  double sigma0;            // base shift (smallest sigma)
  double ds[NPMAX];         // sigma_i - sigma_0, ascending
  double omega[NPMAX];
  double gbound[NPMAX];     // max over [a,b] of x / (x^2 + sigma_i)
};

// Launch shape for a site x rhs kernel.
struct Shape {
  int nsb;   // site blocks
  int by;    // rhs per block
  int ngr;   // rhs groups
  dim3 grid() const { return dim3((unsigned)(nsb * ngr)); }
  dim3 block() const { return dim3(BX, by); }
};
Shape make_shape(int V, int nrhs);
// the lattice is covered by whole tiles of Wilson-kernel variant 2
bool wilson_tiles_fit(const Geom& g);

// ---------------------------------------------------------------- Wilson kernel
// K in (Sec. 1) with optional per-(rhs, block) partials {||out||^2, ||in||^2}.
// ms (may be null): skip systems whose multi-shift solve is done.
void launch_wilson_K(int pin, int plink, int pout, const Geom& g, double kappa, LinkRef links,
                     SpinorRef in, SpinorRef out, int nrhs, double* partials, const MsRhs* ms,
                     cudaStream_t st);
// Multi-shift CG second half: Ap = K in + sigma0 p;  r -= alpha Ap; partials {||r||^2}.
void launch_wilson_mscg_r(int pt, int plink, int pr, int pp, const Geom& g, double kappa, LinkRef links,
                          SpinorRef t, SpinorRef p0, SpinorRef r, int nrhs, double sigma0,
                          double* partials, const MsRhs* ms, cudaStream_t st);
// out = c1 v + c2 (y - kappa hop y)  [= c1 v + c2 gamma5 K y], optionally times gamma5,
// with optional partials {Re (w, out), Im (w, out), ||out||^2, ||w||^2}. coef (device,
// may be null) holds per-rhs (c1, c2) pairs that replace c1, c2.
void launch_wilson_ovl(int py, int plink, int pv, const Geom& g, double kappa, LinkRef links, SpinorRef y,
                       SpinorRef v, SpinorRef out, SpinorRef w, int nrhs, double c1, double c2,
                       const double* coef, int herm, double* partials, cudaStream_t st);

// Stored-basis Lanczos, the two Wilson launches of one iteration. The basis W is a batch
// of cap * nrhs fields, field l * nrhs + rhs holding W_l of system rhs; lz[rhs].j selects
// the slot, so that one captured graph serves every iteration.
//   K mode: t = (1 / n_j) K W_j, partials {||t||^2} (alpha_j = ||K v_j||^2);
//   L mode: W_{j+1} = K t - a W_j - b W_{j-1}, partials {||W_{j+1}||^2}.
// The scalar step of each system runs inside the same launch: every block writes its
// partial sums and counts itself in ctr[rhs]; the block that arrives last sums the
// partials in a fixed order and updates the system's state (K mode: alpha_j, a, b; L mode:
// beta_j, every pole's pivot and residual, the stopping test), then resets ctr[rhs].
struct LzCtl {
  LzRhs* lz;
  unsigned int* ctr;   // per system, zero between launches
  double* ahist;       // alpha_j, nrhs rows of hcap
  double* bhist;       // beta_j
  int hcap;
  const Poles* poles;
};
void launch_wilson_lzK(int pw, int plink, int pt, const Geom& g, double kappa, LinkRef links, SpinorRef W,
                       SpinorRef t, int nrhs, double* partials, const LzCtl& ctl, cudaStream_t st);
void launch_wilson_lzL(int pt, int plink, int pw, const Geom& g, double kappa, LinkRef links, SpinorRef t,
                       SpinorRef W, int nrhs, double* partials, const LzCtl& ctl, cudaStream_t st);
// W_0 = v (precision conversion), y = 0, partials {||W_0||^2}
void launch_lz_init(int pv, int pw, int py, SpinorRef v, SpinorRef W, SpinorRef y, int nrhs, int V,
                    double* partials, cudaStream_t st);
// start a cycle from the norm partials of W_0; first = 1: weights omega_i, budget eta ||W_0||
void launch_lz_start(LzRhs* lz, const double* partials, int nsb, int nrhs, const Poles* poles,
                     const double* eta, int maxit, int cap, int first, cudaStream_t st);
// coefficients of the stored vectors in y = sum_i w_i x_i (per system, cap doubles) from
// the tridiagonal solves; Y is scratch of nrhs * npoles * 2 cap doubles. For a system whose
// cycle filled up, the weights of the next cycle are set too.
void launch_lz_coef(LzRhs* lz, const double* ahist, const double* bhist, int cap, const Poles* poles, double* Y,
                    double* coefW, int nrhs, cudaStream_t st);
// y += sum_l coefW[l] W_l for every system with basis vectors this cycle
void launch_lz_combine(int pw, int py, SpinorRef W, SpinorRef y, const double* coefW, const LzRhs* lz, int cap,
                       int nrhs, int V, cudaStream_t st);
// systems whose cycle filled up: W_0 = W_j, partials {||W_0||^2} (others zero)
void launch_lz_restart(int pw, SpinorRef W, const LzRhs* lz, int nrhs, int V, double* partials, cudaStream_t st);

// ---------------------------------------------------------------- multi-shift CG
void launch_ms_init(int pv, int pr, int pp, SpinorRef v, SpinorRef r, SpinorRef pbase, SpinorRef y,
                    int npoles, int nrhs, int V, double* partials, cudaStream_t st);
void launch_ms_scalar0(MsRhs* ms, const double* partials, int nsb, int nrhs, const Poles* poles,
                       const double* eta_abs /* per rhs, relative eta */, int maxit, cudaStream_t st);
void launch_ms_scalar1(MsRhs* ms, const double* partials, int nsb, int nrhs, const Poles* poles,
                       cudaStream_t st);
void launch_ms_scalar2(MsRhs* ms, const double* partials, int nsb, int nrhs, const Poles* poles,
                       cudaStream_t st);
void launch_ms_update(int pr, int pp, SpinorRef r, SpinorRef pbase, SpinorRef y, int npoles, int nrhs,
                      int V, const MsRhs* ms, cudaStream_t st);
// Variant that keeps every shifted solution: x_i += alpha_i p_i (x: npoles * nrhs fields,
// index i * nrhs + rhs, FP64), used by the gauge-link gradient.
void launch_ms_update_x(SpinorRef r, SpinorRef pbase, SpinorRef xs, int npoles, int nrhs, int V, const MsRhs* ms,
                        cudaStream_t st);

// ---------------------------------------------------------------- vector kernels
// Canonical interleaved complex (c128 / c64) <-> internal layout.
void launch_pack(int dtype, const void* canon, int pout, SpinorRef out, int nrhs, int V, cudaStream_t st);
void launch_unpack(int dtype, void* canon, int pin, SpinorRef in, int nrhs, int V, cudaStream_t st);
// Precision conversion between internal fields.
void launch_convert(int pin, SpinorRef in, int pout, SpinorRef out, int nrhs, int V, cudaStream_t st);
// Per-rhs complex scalars a[rhs], b[rhs] (device, interleaved re/im):
//   z = a x + b y       (z may alias x or y)
void launch_axpby(int p, const double* a, const double* b, SpinorRef x, SpinorRef y, SpinorRef z,
                  int nrhs, int V, cudaStream_t st);
// partials {Re, Im} of (x, y) per (rhs, block)
void launch_dot(int px, SpinorRef x, int py, SpinorRef y, int nrhs, int V, double* partials, cudaStream_t st);
// partials {||x||^2, 0}
void launch_norm2(int px, SpinorRef x, int nrhs, int V, double* partials, cudaStream_t st);
// Sum partials over blocks per rhs in a fixed order: out[rhs*NVRED + j], j < NVRED.
void launch_reduce_partials(const double* partials, int nsb, int nrhs, double* out, cudaStream_t st);
// x = gamma5 x
void launch_gamma5(int p, SpinorRef x, int nrhs, int V, cudaStream_t st);
void launch_zero(int p, SpinorRef x, int nrhs, int V, cudaStream_t st);

// SUMR step (Alg. 1 basis + progressive Givens QR of rho + B, Sec. 2 / App. A).
// sc (device) per rhs: 9 complex scalars
//   0 Rm1 (R_{j-1,j}), 1 gs (gamma_j sigma_{j-1}), 2 invRjj, 3 sigma_{j-1}, 4 z_{j-1},
//   5 g_j, 6 gamma_j, 7 1/sigma_j, 8 sigma_j
// pnew = (q - Rm1 p + gs S) invRjj; S = sig_{j-1} S + z p; p = pnew; x += g p;
// qn = (u + gamma q~) / sigma_j; q~ = sigma_j q~ + conj(gamma) qn; q = qn.
// active (device int per rhs) = 0 freezes that system. partials {||q||^2}.
void launch_sumr_update(int p, const double* sc, const int* active, SpinorRef x, SpinorRef q, SpinorRef qt,
                        SpinorRef pv, SpinorRef S, SpinorRef u, int nrhs, int V, double* partials,
                        cudaStream_t st);

// Multi-mass SUMR step: nm masses share the basis of each of ns sources (system k ns + j);
// sc holds 18 doubles per system (as above), scq 6 per source (gamma, 1/sigma, sigma);
// active per system, qactive per source. partials {||q||^2} per source.
void launch_sumr_mm_update(int p, const double* sc, const double* scq, const int* active, const int* qactive,
                           SpinorRef x, SpinorRef q, SpinorRef qt, SpinorRef pv, SpinorRef S, SpinorRef u, int ns,
                           int nm, int V, double* partials, cudaStream_t st);

// ---------------------------------------------------------------- dense blocks
// G[i, j] += (A_i, B_j) for i < na, j < nb (complex, FP64 accumulation); A and B are
// batches of na / nb spinors; G is na x nb row-major complex (interleaved). Partials
// per block are reduced in a fixed order.
void launch_gram(int pa, SpinorRef A, int na, int pb, SpinorRef B, int nb, int V, double* G,
                 double* work, size_t work_doubles, int g5, cudaStream_t st);
// The same block on the tensor cores, FP64-accurate (operands split into 7-bit digits with
// exact BF16 products and exact FP32 sums; P64 and P32 fields only). ex: na + nb ints;
// partial: tc_gram_work_doubles(na, nb, nsplit) doubles; err set to 1 on a bounded wait that
// gave up.
bool tc_gram_supported(int pa, int pb);
int tc_gram_splits(int na, int nb, int V, int nsm);
size_t tc_gram_work_doubles(int na, int nb, int nsplit);
void launch_tc_gram(int pa, const void* A, int na, int pb, const void* B, int nb, int V, int g5, int nsplit,
                    double* G, double* partial, int* ex, int* err, cudaStream_t st);
// Y_j (+)= sum_i A_i C[i, j] for j < ny (C na x ny row-major complex, device); Y distinct
// from A. add = 1 accumulates into Y.
void launch_combine(int pa, SpinorRef A, int na, const double* C, int py, SpinorRef Y, int ny, int V, int add,
                    cudaStream_t st);

// ---------------------------------------------------------------- force
// G[s][mu] += sum_i coef_i (-kappa/2) (conj(F) + G^T) for the three terms of the
// Zolotarev derivative (see force.cu); psi FP64 (1 field), a, Ka, b, Kb FP64 (npoles fields).
void launch_force(int fp32, const Geom& g, double kappa, SpinorRef psi, SpinorRef a, SpinorRef Ka, SpinorRef b,
                  SpinorRef Kb, int npoles, const double* coef /* device, npoles */, double* G, cudaStream_t st);

}  // namespace ovl
