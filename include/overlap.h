/*
 * overlap.h -- C ABI of liboverlap, a GB300 (sm_103a) implementation of the
 * deflated overlap-fermion inverter of Cundy & Lee, "The eigSUMR inverter for
 * overlap fermions" (arXiv:1501.01855).
 *
 * Operators (Sec. 1):
 *   K      = gamma5 [1 - kappa sum_mu ((1-gamma_mu) U_mu(x) T_{+mu} + (1+gamma_mu) U_mu(x-mu)^dag T_{-mu})],
 *            kappa = 1/(8 - 2 m0)                       (Sec. 1, the equation for aK_xy)
 *   D(mu)  = 1/2 (1 + mu + (1 - mu) gamma5 sign(K))      (Sec. 1)
 *   sign(K) ~ eps(K) = sum_i omega_i K (K^2 + sigma_i)^-1 (Zolotarev, Sec. 3),
 *            evaluated by multi-shift CG to a caller-chosen accuracy eta.
 * Solvers: GMRESR (Alg. 3) around relaxed SUMR (Algs. 1-2, Sec. 3) or relaxed,
 * spectrally preconditioned CGNE (Alg. 4); eigSUMR accumulation (Algs. 5-6);
 * Galerkin / least-squares deflation (Sec. 4).
 *
 * Conventions shared by every entry point
 *   - Every call returns an ovl_status; on failure overlap_last_error() gives a
 *     one-line reason. Nothing aborts the process.
 *   - Lattice dims are {Lx, Ly, Lz, Lt}; site = ((t*Lz + z)*Ly + y)*Lx + x.
 *   - Spinors are in the canonical layout [site][spin 4][colour 3] of interleaved
 *     complex numbers, either complex128 (OVL_C128) or complex64 (OVL_C64).
 *     A batch of n spinors is n such fields back to back.
 *   - Links are [site][mu 4][row 3][col 3] complex128, mu = 0..3 -> x,y,z,t.
 *   - The gamma matrices are the Hermitian chiral (DeGrand-Rossi) set, gamma5 =
 *     diag(1,1,-1,-1).
 *   - "on_device" = 1: the pointers are CUDA device pointers on the context's
 *     device; 0: host pointers. Page-locked host buffers (cudaHostAlloc,
 *     cudaHostRegister) are copied by DMA directly; pageable ones go through the
 *     context's pinned staging buffer.
 *   - The library never frees or keeps caller memory. All internal memory is
 *     owned by the context (or the deflation object) and released by the
 *     matching destroy call.
 *   - All work is issued on the context's stream (ovl_params.stream, default
 *     the legacy default stream); calls return after that work has completed.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef OVERLAP_H
#define OVERLAP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ovl_ctx ovl_ctx;
typedef struct ovl_defl ovl_defl;

typedef enum {
  OVL_OK = 0,
  OVL_EINVAL = -1,      /* bad argument (null pointer, bad size, bad enum)            */
  OVL_ENOMEM = -2,      /* device or host allocation failed                           */
  OVL_ECUDA = -3,       /* a CUDA runtime call failed (message has the CUDA error)    */
  OVL_ENOCONV = -4,     /* iteration limit reached before the tolerance               */
  OVL_EBREAKDOWN = -5,  /* SUMR/CG breakdown (sigma_j^2 <= 0, NaN or Inf)             */
  OVL_EAPPROX = -6,     /* Zolotarev Delta(n_poles, a, b) > eps_sign                  */
  OVL_ETIMEOUT = -7     /* a device-side bounded wait gave up                         */
} ovl_status;

enum { OVL_C128 = 0, OVL_C64 = 1 };                     /* spinor element types       */
/* OVL_PREC_F64E: FP64-accurate double-float ("hi + lo" of two floats, ~47-bit significand)
 * computed on the FP32 pipes; storage the size of FP64. */
enum { OVL_PREC_F64 = 0, OVL_PREC_F32 = 1, OVL_PREC_F16 = 2, OVL_PREC_F64E = 3, OVL_PREC_AUTO = -1 };
enum { OVL_SOLVER_SUMR = 0, OVL_SOLVER_CG = 1 };

typedef struct {
  int    solver;        /* OVL_SOLVER_SUMR (GMRESR(relSUMR)) or OVL_SOLVER_CG (GMRESR(relCG))   */
  int    mixed;         /* 1: low-precision sign when eta allows (Sec. 3, mixed precision);
                           0: plain FP64 everywhere                                              */
  int    half_storage;  /* 1: FP16 links/vectors in the sign when eta >= half_switch            */
  int    emulate_fp64;  /* 1: accurate signs (eta < sp_switch, or mixed = 0) in double-float on
                           the FP32 pipes (OVL_PREC_F64E; GB300 runs FP64 at 1/60 of its FP32
                           rate); 0: native FP64. Default 1                                  */
  double eta_floor;     /* sign accuracy never worse than this (Sec. 3): default 1e-2           */
  double sp_switch;     /* eta above which the FP32 sign is used: default 1e-6                  */
  double half_switch;   /* eta above which FP16 storage is used: default 2e-3                    */
  double eta_precond;   /* middle-solve relative accuracy eta~ (Alg. 3); 0 = tol^(1/3)          */
  double relax_factor;  /* relaxation eta_j = relax_factor * eps_A ||b|| / ||r_j||: default 1   */
  int    gmresr_max;    /* outer steps, default 30                                              */
  int    inner_max;     /* middle-solver iterations per outer step, default 2000                */
  int    mscg_max;      /* multi-shift CG iterations per sign, default 5000                     */
  double delta_split;   /* pair splitting delta of Sec. 5, default 0.01                         */
  double c_spec;        /* spectral-preconditioner constant c (Sec. 4), default sqrt(3)/2      */
  int    bc_t;          /* 0 periodic, 1 antiperiodic in t (fermions only)                      */
  double a_override;    /* >0: use this lower bound a of |lambda(K)|, else estimate by Lanczos  */
  double b_override;    /* >0: use this upper bound b of |lambda(K)|, else estimate by Lanczos  */
  int    batch_max;     /* systems advanced together in one lock-step batch, default 36         */
  int    wilson_variant;/* Wilson-kernel launch shape: -1 autotune at create (default), 0 one
                           thread per site, 1 four threads per site (one per direction), 2 one
                           thread per site on 8x4x4x2 tiles (needs extents divisible by those),
                           3 two threads per site, one per half spinor (double-float only; the
                           other precisions use 0)                                           */
  int    use_graphs;    /* 1 (default): run the multi-shift CG iterations as cached CUDA graphs
                           (not while profiling); 0: launch every kernel on the stream        */
  int    verify;        /* 1: after a solve, recompute ||b - D x|| / ||b|| with an FP64 sign at
                           eps_sign (one more sign application per system); 0: report the
                           GMRESR recursive residual. Default 1                                 */
  int    sign_method;   /* how the Zolotarev sum (Sec. 3) is evaluated: 0 (default) Lanczos on
                           K^2 with its basis stored in HBM (one vector per step; every pole's
                           solution from a tridiagonal solve and one pass over the basis), when
                           the basis of a batch fits in basis_gb (else as 1); 1 multi-shift CG
                           (one search direction per pole, updated every step); 2 stored-basis
                           Lanczos always (sub-batched to fit basis_gb)                        */
  double basis_gb;      /* device memory for stored Lanczos bases, GB, default 96              */
  int    multimass;     /* 1 (default): in undeflated GMRESR(relSUMR) solves of several masses,
                           batch by source and let the masses of a source share one SUMR basis
                           (and one sign application per step) in the first middle solve, which
                           starts from r = b for every mass (Sec. 2: SUMR adapts to many shifts);
                           0: every system runs its own SUMR                                   */
  int    force_pole_group;/* overlap_force: >0 solve the shifted systems of this many poles at a
                           time (their solutions recomputed per group instead of all stored);
                           0 (default): all poles at once when their fields fit in half the free
                           device memory, else as many as fit                                */
  int    lanczos_cap;   /* >0: at most this many basis vectors per Lanczos cycle (a full cycle
                           restarts from its last vector, to which every pole's residual is
                           parallel); 0 (default): sized from the steps this context has
                           needed at that accuracy, else from the CG bound of the base shift */
  int    gram_method;   /* dense blocks (Gram matrices of the Ritz step, Alg. 6, and the
                           projections of the deflated starts, Sec. 4): 0 (default) on the
                           tensor cores with FP64-level accuracy (operands split into six
                           7-bit digits, exact BF16 products, exact FP32 sums over 512 reals,
                           double-float and FP64 above) for FP64 and FP32 fields, else as 1;
                           1 CUDA-core kernel with FP32 products and FP64 sums              */
  void*  stream;        /* cudaStream_t for all work; NULL = legacy default stream              */
} ovl_params;

typedef struct {
  int    converged;        /* 1 if the FP64 true residual met tol                                */
  int    outer_iters;      /* GMRESR steps                                                       */
  int    inner_iters;      /* SUMR or CG iterations summed over outer steps                      */
  int    sign_calls;       /* applications of the sign function                                  */
  long long wilson_calls;  /* Wilson-kernel applications, FP64 counted as 2 (Sec. 6)             */
  long long wilson_f64, wilson_f32, wilson_f16;   /* raw counts per precision                   */
  double true_residual;    /* ||b - D x|| / ||b||: with params.verify, recomputed with an accurate
                              sign (double-float, or FP64 when emulate_fp64 = 0) at accuracy
                              min(eps_sign, 0.1 tol mu); else the GMRESR recursive residual      */
  double seconds;          /* wall time of this system's solve (shared by a batch)               */
} ovl_solve_info;

/* Fill *p with the defaults listed above. */
ovl_status ovl_params_default(ovl_params* p);

/* Build a context for one gauge field (the device current at the call).
 *   ctx       receives the new context (caller frees it with overlap_destroy).
 *   dims[4]   {Lx, Ly, Lz, Lt}, each even and >= 2.
 *   links     host, canonical layout, complex128, 4*9*V entries; copied (the caller
 *             keeps ownership) into the library's device layouts: 12-real FP64 / FP32 /
 *             FP16 copies (row 3 of every SU(3) link rebuilt as conj(row1 x row2) in
 *             registers) and an 18-real double-float copy with one slot per hop.
 *   m0        Wilson mass, kappa = 1/(8 - 2 m0) (Sec. 1).
 *   mu        default overlap mass parameter of D(mu) (Sec. 1).
 *   n_poles   Zolotarev order N_Z (Sec. 3), 1..64.
 *   eps_sign  required Zolotarev Delta; OVL_EAPPROX if the bounds [a, b] need more
 *             poles than n_poles.
 *   params    may be NULL (defaults).
 * The spectral bounds a = min|lambda(K)|, b = max|lambda(K)| come from
 * params->a_override / b_override when positive, else from an FP64 Lanczos run
 * on K^2 with safety margins (a * 0.95, b * 1.05). Create also times the Wilson-kernel
 * launch shapes (autotuner, see ovl_wilson_tuning). Errors: OVL_EINVAL (bad sizes,
 * m0 outside (0, 4), mu outside [0, 1)), OVL_EAPPROX, OVL_ENOMEM, OVL_ECUDA; *ctx is
 * then NULL. */
ovl_status overlap_create(ovl_ctx** ctx, const int dims[4], const double* links, double m0, double mu,
                          int n_poles, double eps_sign, const ovl_params* params);
/* Free every device and host resource of the context (NULL is allowed). Deflation
 * spaces made with it must be destroyed first. */
void overlap_destroy(ovl_ctx* ctx);
/* One-line reason of the last failed call on ctx ("" if none); valid until the next
 * call on the same context. */
const char* overlap_last_error(const ovl_ctx* ctx);

/* Release the device memory the context caches between calls: every workspace (solver
 * vectors, multi-shift pole vectors, the stored Lanczos basis) and the captured CUDA
 * graphs. The gauge field, the Zolotarev data and deflation spaces stay; the next call
 * allocates what it needs again. Synchronises the context stream. */
ovl_status ovl_trim(ovl_ctx* ctx);

/* Host-only (no GPU needed): the Zolotarev rational of order n on a < |x| < b
 * (Sec. 3), eps(x) = sum_i omega_i x / (x^2 + sigma_i), sigma ascending, and its
 * maximum error delta, from Jacobi elliptic functions (AGM / descending Landen). */
ovl_status ovl_zolotarev_coeffs(int n, double a, double b, double* omega, double* sigma, double* delta);

/* Host-only (no GPU, no context): the small dense FP64 numerics that the solvers run on
 * the host between kernel launches, exported so that they can be checked on their own.
 * Complex matrices are n x n, row-major, interleaved (re, im) doubles; inputs are read
 * only, outputs are caller buffers of the same size; 1 <= n <= 4096, else OVL_EINVAL.
 *   ovl_host_eigh             Hermitian eigendecomposition (Householder reduction to a
 *                             real tridiagonal, implicit QR steps with Wilkinson shifts;
 *                             cyclic Jacobi rotations should those not converge):
 *                             w ascending, z the orthonormal eigenvectors as
 *                             columns (a = z diag(w) z^dag). The diagonalisation of
 *                             L^-1 M U^-1 in the Ritz step (Alg. 6), of the projected
 *                             gamma5 D in the least-squares start (Sec. 4) and of the
 *                             Rayleigh quotient in the kernel low-mode deflation (Sec. 1).
 *                             The full matrix is read; a non-finite entry gives OVL_EINVAL.
 *   ovl_host_cholesky         a = l l^dag with l lower triangular, positive real diagonal
 *                             (the E = U^dag U of Alg. 6); OVL_EBREAKDOWN unless a is
 *                             numerically positive definite.
 *   ovl_host_lower_inverse    li = l^-1 for lower-triangular l (zero entries above the
 *                             diagonal are not read); OVL_EBREAKDOWN on a zero pivot.
 *   ovl_host_lu_solve         x = a^-1 b for nb right-hand sides (b, x: n x nb row-major)
 *                             by partially pivoted LU (the least-squares normal equations
 *                             of the deflated start, Sec. 4); OVL_EBREAKDOWN when a pivot
 *                             column is exactly zero.
 *   ovl_host_tridiag_extremes smallest and largest eigenvalue of the real symmetric
 *                             tridiagonal matrix (diagonal d[n], off-diagonal e[n-1]; e
 *                             unused for n = 1) by Sturm-sequence bisection from the
 *                             Gershgorin interval: the extremes of the Lanczos tridiagonal
 *                             of K^2, whose square roots estimate the interval [a, b] of
 *                             |K| that the rational of Sec. 3 covers. */
ovl_status ovl_host_eigh(int n, const double* a, double* w, double* z);
ovl_status ovl_host_cholesky(int n, const double* a, double* l);
ovl_status ovl_host_lower_inverse(int n, const double* l, double* li);
ovl_status ovl_host_lu_solve(int n, const double* a, const double* b, int nb, double* x);
ovl_status ovl_host_tridiag_extremes(int n, const double* d, const double* e, double* lmin, double* lmax);

/* Host-only: one step of the library's relSUMR recurrence for one system (Algs. 1-2, Sec. 2;
 * the short recurrence re-derived from App. A: progressive Givens QR of rho I + B^), as the
 * solver runs it between the sign application u = V q_j with its fused reductions and the
 * vector update. rho = (1 + mu)/(1 - mu) > 1; dots = {Re (q~_j, u), Im (q~_j, u), ||u||^2,
 * ||q~_j||^2} with (a, b) = sum conj(a) b. state[11], in and out: {gamma_{j-1} (re, im),
 * s_{j-1} (re, im), c_{j-1}, sigma_{j-1}, zeta (re, im), g^ (re, im), j}; a solve starts from
 * {0, 0, 0, 0, 1, 0, 1, 0, ||r_0||, 0, 0} with q_0 = q~_0 = r_0 / ||r_0||, p = S = 0. coef[18]
 * receives 9 complex numbers (R, gs, iR, sp, z, g, gamma_j, 1/sigma_j, sigma_j) for the update
 *   p' = (q_j - R p + gs S) iR,  S <- sp S + z p,  p <- p',  x <- x + g p',
 *   q_{j+1} = (u + gamma_j q~_j) / sigma_j,  q~_{j+1} = sigma_j q~_j + conj(gamma_j) q_{j+1},
 * after which |g^| is the residual estimate ||b - (rho + V) x||. OVL_EBREAKDOWN, state
 * untouched, when sigma_j^2 vanishes to rounding (an exhausted Krylov space) or a dot is not
 * finite; OVL_EINVAL for rho <= 1, a null pointer or a non-finite state. */
ovl_status ovl_host_sumr_step(double rho, const double* dots, double* state, double* coef);

/* Host-only: the deflated start of relSUMR (Sec. 4) from Gram blocks, as the solver runs it
 * after computing them on the device: for a space psi_1 .. psi_n with w_i = gamma5 eps(K) psi_i
 * (so that D(mu) psi = (1+mu)/2 psi + (1-mu)/2 w), VV = (psi_i, psi_j), WW = (w_i, w_j),
 * WV = (w_i, psi_j), G5VV = (psi_i, gamma5 psi_j), G5VW = (psi_i, gamma5 w_j) (n x n) and, for
 * nsys right-hand sides b_j at masses mus[j], VB = (psi_l, b_j) and WB = (w_l, b_j) (n x nsys),
 * all complex, row-major, interleaved. The space is rotated to psi' = psi Y diagonalising
 * (psi'_i, gamma5 D psi'_j); alpha minimises ||b - D psi' alpha|| (per_vector = 1: the
 * per-vector alpha_j = (D psi'_j, b) / (D psi'_j, D psi'_j) of Sec. 4 instead). coefs
 * (n x nsys) receives x0 = psi coefs_j. OVL_EBREAKDOWN for singular normal equations,
 * OVL_EINVAL for n outside 1..1024, nsys outside 1..4096, a mass outside (0, 1), a null
 * pointer or a non-finite entry. */
ovl_status ovl_host_defl_start(int n, const double* VV, const double* WW, const double* WV, const double* G5VV,
                               const double* G5VW, int nsys, const double* VB, const double* WB, const double* mus,
                               int per_vector, double* coefs);

/* Host-only: the k x k algebra of one Ritz step (Alg. 6) as the eigen accumulation runs it
 * between its Gram blocks and the rotation of the basis, for a basis v_1 .. v_k with
 * v^D_i = D(mu) v_i (Sec. 5). E = (v_i, v_j), MVD = (v^D_i, v^D_j), G5 = (v_i, gamma5 v^D_j):
 * k x k complex, row-major, interleaved (re, im). Cholesky E = U^dag U (or, without a factor
 * or with a pivot below 1e-10 of E's largest diagonal, the eigendecomposition of E with
 * directions below 1e-10 of its largest eigenvalue dropped), eigenvectors Y of
 * U^-dag (MVD + 2 mu delta G5) U^-1, the lowest keep kept. restart = 1 is the locally
 * optimal restart of a full basis (on the Cholesky path): the lowest keep Ritz vectors of
 * the basis and of the basis without v_k, Rayleigh-Ritz on their span (keep to 2 keep pairs;
 * near-duplicates of the two sets are dropped). Out: *kept, the Ritz values ritz (ascending; D^dag D + 2 mu delta gamma5 D),
 * the coefficients C (k x *kept complex, row-major) of the Ritz vectors in v_1 .. v_k and
 * the residual norms ||gamma5 v^D - v (v, gamma5 v^D)|| (res); ritz and res hold 2 keep
 * doubles, C 2 k keep complex numbers. OVL_EINVAL for k outside 1..1024, keep outside 1..k,
 * mu outside (0, 1), delta < 0, a null pointer or a non-finite Gram entry. */
ovl_status ovl_host_ritz(int k, const double* E, const double* MVD, const double* G5, double mu, double delta,
                         int keep, int restart, double* ritz, double* C, double* res, int* kept);

/* Zolotarev data of the context: omega[n], sigma[n] (may be NULL; n the pole count in use:
 * n_poles at create, or the count ovl_kernel_deflate chose),
 * the error Delta and the bounds a, b actually used (Sec. 3). */
ovl_status overlap_zolotarev(const ovl_ctx* ctx, double* omega, double* sigma, double* delta,
                             double* a, double* b);

/* out = K in for n spinors (Sec. 1); in and out may not alias. prec selects the kernel:
 * OVL_PREC_F64 computes in FP64, OVL_PREC_F64E in double-float, OVL_PREC_F32 / F16
 * round the input to FP32 / FP16 storage and compute in FP32. OVL_EINVAL for a null
 * pointer, n < 1 or an unknown dtype / prec. */
ovl_status ovl_wilson_apply(ovl_ctx* ctx, const void* in, void* out, int n, int dtype, int on_device,
                            int prec);

/* out = K in, like ovl_wilson_apply, for callers that cannot let the library allocate
 * device memory during the call: code whose device memory belongs to its own pool or
 * sits under a hard cap, and loops that must not stall in the allocator. (The paper
 * has no counterpart; this is a property of the library, not of the method.)
 *   in, out  device pointers (the context's device must be current), n canonical
 *            spinors each; dtype as for ovl_wilson_apply, prec OVL_PREC_F64, F32 or F16
 *            (anything else returns OVL_EINVAL).
 * The two layout-conversion buffers live in one static device array of
 * OVL_NOALLOC_BYTES (48 MiB) that every device loading the library holds until the
 * process exits. A call needs 2 n V x 192 bytes in FP64, x 96 in FP32 and x 52 in FP16
 * (48 bytes of spinor plus a 4-byte scale per site), each buffer rounded up to 256
 * bytes, so n V <= 131072 in FP64; a larger call returns OVL_EINVAL. No cudaMalloc,
 * cudaFree or other allocating routine is called. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) once; make that first call before
 * any stream capture begins. Like every entry point here,
 * the call returns after its work on the context stream has completed. All calls share
 * the array: calls that overlap on the GPU race on it, and it keeps the last call's
 * intermediate data (nothing in it has to start at zero). */
#define OVL_NOALLOC_BYTES ((size_t)48 << 20)
ovl_status ovl_wilson_apply_noalloc(ovl_ctx* ctx, const void* in, void* out, int n, int dtype, int prec);

/* out = eps(K) in (Sec. 3) for n spinors, multi-shift CG stopped at accuracy eta
 * (the per-pole rule of the Zolotarev sum; eta <= 0 means eps_sign). prec as above,
 * OVL_PREC_AUTO picks by eta. OVL_ENOCONV when a system reached params.mscg_max
 * iterations before eta was met (the message names the system), OVL_EBREAKDOWN on a
 * non-positive or non-finite curvature; every solver that applies the sign passes
 * these on. */
ovl_status ovl_sign_apply(ovl_ctx* ctx, const void* in, void* out, int n, int dtype, int on_device,
                          double eta, int prec);

/* out = D(mu) in (Sec. 1) for n spinors at sign accuracy eta (eta <= 0: eps_sign).
 * hermitian = 1 returns H in = gamma5 D(mu) in instead. */
ovl_status overlap_apply(ovl_ctx* ctx, double mu, const void* in, void* out, int n, int dtype,
                         int on_device, double eta, int prec, int hermitian);

/* The middle solver alone: relaxed SUMR (Algs. 1-2, Sec. 3) for D(mu) x = b, n systems,
 * stopped at the relative residual estimate tol or after maxit iterations. eta_fixed > 0
 * applies the sign at that accuracy every iteration; eta_fixed <= 0 relaxes it as
 * eta_j = tol ||b|| / ||r_j|| (never worse than params.eta_floor). hist (may be NULL)
 * receives maxit * n residual estimates ||r_j|| / ||b|| (system-major, 0 after the
 * last iteration); iters (may be NULL) the iteration count per system. */
ovl_status overlap_sumr(ovl_ctx* ctx, double mu, const void* b, void* x, int n, int dtype, int on_device, double tol,
                        double eta_fixed, int maxit, double* hist, int* iters);

/* Solve D(mu_k) x = b for nrhs sources and nmass masses (GMRESR, Alg. 3, around
 * relSUMR or relCG, Sec. 3). x holds nmass*nrhs spinors, mass-major
 * (x[k*nrhs + j] solves mass k, source j). tol is the relative FP64 true-residual
 * target. defl may be NULL (undeflated) or a space from eigsumr_accumulate();
 * its eigenvectors of D^dag D are mass independent (Sec. 1) and serve every mass.
 * info (may be NULL) receives nmass*nrhs records. Systems are advanced in
 * lock-step batches of at most params.batch_max. */
ovl_status overlap_solve(ovl_ctx* ctx, int nrhs, const double* mus, int nmass, const void* rhs, void* x,
                         int dtype, int on_device, double tol, ovl_defl* defl, ovl_solve_info* info);

/* Solve D(mu) x = b once while accumulating Ritz vectors of D^dag D + 2 mu delta H
 * (Algs. 5-6, Sec. 5) with basis size m_basis, keeping n_eig, on the Krylov vectors of the
 * context's middle solver: eigSUMR (params.solver = OVL_SOLVER_SUMR: q_j and V q_j of
 * Alg. 5) or eigCG (OVL_SOLVER_CG: the residual directions of relCG and D applied to them,
 * from vectors the CG step computes anyway). If *defl is
 * NULL a new space is created; otherwise its vectors seed the basis and are
 * improved. The space can then be passed to overlap_solve(). OVL_ENOCONV: the solve
 * stopped short of tol; the space is still built (or refined) and *defl set, and x
 * holds the last iterate. */
ovl_status eigsumr_accumulate(ovl_ctx* ctx, ovl_defl** defl, int n_eig, int m_basis, double mu,
                              const void* rhs, void* x, int dtype, int on_device, double tol,
                              ovl_solve_info* info);

/* Standalone eigensolver (Sec. 6): approximate eigenvectors of D^dag D (and of gamma5 D)
 * at mass mu from the eigSUMR Arnoldi process (Alg. 1 on V = gamma5 eps(K), Algs. 5-6) run
 * without a linear solve, for callers who want the deflation space first (or a better one
 * than the accumulation during solves gives). Rounds of round_diags Ritz steps (the paper
 * used 24): each round ends with a Rayleigh-Ritz step over its vectors and those kept at
 * the previous two rounds, an accurate recomputation of v^D, and a restart from the last
 * basis vector orthogonalised against the current ones (also when ||q|| - 1 exceeds 0.1).
 * The sign accuracy follows the Sec. 5.1 bound.
 *   defl      in/out: NULL creates a space of n_eig vectors, else it is improved.
 *   m_basis   Arnoldi basis, >= 2 n_eig + 8 (at a basis restart 2 n_eig vectors are kept).
 *   start     one canonical spinor (dtype, on_device), or NULL for a Z2 source.
 *   max_steps budget of sign applications; res_tol: stop once every residual
 *             ||gamma5 D psi - psi (psi, gamma5 D psi)|| is at most this.
 *   steps_done (may be NULL) receives the sign applications used. */
ovl_status ovl_eigensolve(ovl_ctx* ctx, ovl_defl** defl, int n_eig, int m_basis, double mu, const void* start,
                          int dtype, int on_device, int max_steps, double res_tol, int round_diags, int* steps_done);

/* The Ritz recalculation of Alg. 6 (Sec. 5) on a caller-given basis: m spinors v and
 * their v^D = D(mu) v (canonical, dtype and on_device as everywhere; m * 12 V entries
 * each). E = V^dag V is Cholesky-factorised (E = U^dag U; if V has lost linear
 * independence, orthonormalised through the eigendecomposition of E instead), M =
 * (V^D)^dag V^D + 2 mu delta V^dag gamma5 V^D, and the eigenvectors Y of L^-1 M U^-1
 * (ascending) give the new basis V U^-1 Y, of which the lowest n_keep are returned:
 *   v_out, vD_out  n_keep spinors each (new v and v^D; same side and dtype as v);
 *   ritz           host, n_keep Ritz values of D^dag D + 2 mu delta H;
 *   residuals      host, n_keep values ||gamma5 v^D - v (v, gamma5 v^D)|| (may be NULL).
 * The Gram blocks are summed in FP64 from FP32 products, as in the accumulation.
 * OVL_EINVAL for null pointers, m < 1, n_keep outside 1..m, mu outside (0, 1). */
ovl_status ovl_ritz_recalculate(ovl_ctx* ctx, int m, int n_keep, double mu, double delta, const void* v,
                                const void* vD, void* v_out, void* vD_out, int dtype, int on_device, double* ritz,
                                double* residuals);

/* Ritz values (n) and eigenvector residuals ||gamma5 D v - v (v, gamma5 D v)|| (n)
 * of a deflation space; *n receives the number of vectors held; ritz and residuals
 * may be NULL (then only *n is set). */
ovl_status ovl_defl_info(const ovl_defl* defl, int* n, double* ritz, double* residuals);

/* Copy vector i of the space (v_i and v^D_i = D v_i) to host complex128 buffers of
 * 12 V complex entries each (canonical layout; v or vD may be NULL). OVL_EINVAL when
 * i is outside 0..n-1. */
ovl_status ovl_defl_vector(const ovl_defl* defl, int i, double* v, double* vD);

/* Raw little-endian save / load of a deflation space (checkpoint / resume): a text
 * header line "OVLDEFL 1 n=<n> V=<V> mu=<mu>", then per vector v_i and
 * w_i = gamma5 eps(K) v_i as complex128 canonical spinors, then the n Ritz values
 * and n residuals as float64. Load creates a new space on ctx (OVL_EINVAL if the file
 * is malformed or V differs from the context's); save returns OVL_EINVAL when the file
 * cannot be opened or a write fails (the file is then incomplete). Save and load
 * round-trip bit-exactly. */
ovl_status ovl_defl_save(const ovl_defl* defl, const char* path);
ovl_status ovl_defl_load(ovl_ctx* ctx, ovl_defl** defl, const char* path);
/* Free a deflation space (NULL is allowed). */
void ovl_defl_destroy(ovl_defl* defl);

/* Gauge-link gradient of S = phi^dag (D^dag D)^-1 phi through the Zolotarev rational
 * with fixed coefficients (not in the paper; dS = 2 Re sum conj(G) dU).
 *   phi   one canonical spinor (dtype, on_device as everywhere).
 *   dSdU  host, receives 4*9*V complex128 entries (8*9*V doubles) in the canonical
 *         link layout; S (host, may be NULL) receives the action.
 *   tol   accuracy of every inner solve and shifted system.
 * With respect to the links the context was created from. */
ovl_status overlap_force(ovl_ctx* ctx, double mu, const void* phi, int dtype, int on_device, double tol,
                         double* dSdU, double* S);

/* Host-only: the Rayleigh-Ritz step of K inside ovl_kernel_deflate (Sec. 1: the eigenpairs
 * of the Hermitian kernel) on the span of m vectors x_1 .. x_m, from E = (x_i, x_j) and
 * H = (x_i, K x_j) (m x m complex, row-major, interleaved): theta[m], signed, in the order of
 * |theta|, and C (m x m complex, row-major) with X C orthonormal and C^dag H C = diag(theta).
 * OVL_EBREAKDOWN when E has no Cholesky factor; OVL_EINVAL for m outside 1..1024, a null
 * pointer or a non-finite entry. */
ovl_status ovl_host_rayleigh_ritz(int m, const double* E, const double* H, double* theta, double* C);

/* Kernel low-mode deflation of the sign function (Sec. 1: sign(K) = sum_i psi_i psi_i^dag
 * sign(lambda_i); the smallest eigenvectors of K are deflated and the approximation covers
 * the rest of the spectrum). Finds the n_ev eigenpairs of the Hermitian kernel K with the
 * smallest |lambda| to ||K psi - lambda psi|| <= tol (unit psi) by Chebyshev-filtered
 * subspace iteration (at most max_iter filter steps of degree up to 24 on a block of n_ev +
 * max(8, n_ev) FP64 vectors), keeps them in the context, and rebuilds the Zolotarev rational
 * on [a', b] with a' = 0.95 |lambda_min| of K on the complement (300 Lanczos steps on K^2 with
 * the eigenvectors projected out at every step; never below the original a): with
 * n_poles = 0 the fewest poles that keep Delta <= eps_sign, else n_poles (OVL_EAPPROX if
 * that is not enough). From then on every sign application of the context computes
 * sign(K) v = sum_i sign(lambda_i) psi_i (psi_i, v) + eps(K) P v, P = 1 - Psi Psi^dag.
 * n_ev = 0 removes the deflation and restores the context's original interval and poles.
 * overlap_force refuses to run while a deflation is active (it differentiates the rational
 * itself). Outputs (may be NULL): lambda[n_ev] (ascending |lambda|), residual[n_ev], the new
 * lower bound a', the pole count now in use (overlap_zolotarev then reports that many
 * poles), the filter steps taken. OVL_ENOCONV if the eigenpairs did not reach tol within
 * max_iter steps (the context is left undeflated). Allocates 7 (n_ev + guard) FP64 spinor
 * fields of workspace (freed by ovl_trim) and n_ev kept vectors. Synchronises the stream. */
ovl_status ovl_kernel_deflate(ovl_ctx* ctx, int n_ev, double tol, int max_iter, int n_poles, double* lambda,
                              double* residual, double* a_new, int* n_poles_used, int* iters_done);

/* Gram block G[i][j] = (A_i, [gamma5] B_j) = sum over sites and components of
 * conj(A_i) [gamma5] B_j: the dense contraction of the Ritz step (Alg. 6: E = V^dag V,
 * (V^D)^dag V^D, V^dag gamma5 V^D) and of the deflated starts (Sec. 4: Psi^dag b).
 * A: na spinors, B: nb spinors (1 <= na, nb <= 1024) in the canonical layout of dtype
 * (host or device per on_device, read only); they are stored in the library as prec
 * (OVL_PREC_F64 or OVL_PREC_F32) before the contraction. method 0: tensor cores at
 * FP64-level accuracy (the default path of the library's own Gram blocks), 1: CUDA-core
 * kernel with FP32 products and FP64 sums. G: host, na x nb complex128 row-major,
 * overwritten. OVL_ETIMEOUT if a bounded wait inside the tensor-core kernel gave up
 * (the context stays usable). Synchronises the context stream. */
ovl_status ovl_gram(ovl_ctx* ctx, const void* A, int na, const void* B, int nb, int dtype, int on_device,
                    int prec, int g5, int method, double* G);

/* Time `iters` Gram blocks of na x nb random spinors of precision prec held by the
 * library (method as in ovl_gram), back to back on the context stream with CUDA
 * events: *ms_per_call receives the mean milliseconds of one block (its kernels and the
 * memset of its output; no host copy). */
ovl_status ovl_bench_gram(ovl_ctx* ctx, int prec, int na, int nb, int method, int iters, double* ms_per_call);

/* Kernel-level timing collected with CUDA events on the context stream while
 * enabled: per kernel class, launches, total milliseconds and algorithmic bytes.
 * Classes: 0 Wilson FP64, 1 Wilson FP32, 2 Wilson FP16-storage, 3 multi-shift
 * update, 4 vector ops, 5 reductions/scalars, 6 Gram/rotate, 7 force, 8 Wilson
 * double-float. While enabled, the multi-shift iterations are launched one by one
 * (not as CUDA graphs) so that every launch can be timed. */
enum { OVL_PROF_CLASSES = 9 };
ovl_status ovl_profile_enable(ovl_ctx* ctx, int on);
ovl_status ovl_profile_reset(ovl_ctx* ctx);
ovl_status ovl_profile_get(ovl_ctx* ctx, int cls, long long* launches, double* ms, double* bytes);
/* Work units of a class since the last reset: site applications for the Wilson
 * classes (one site of one system through K), site passes for the multi-shift update. */
ovl_status ovl_profile_units(ovl_ctx* ctx, int cls, double* units);

/* Run `iters` back-to-back Wilson-kernel launches on the library's own device
 * fields (n spinors, precision prec) and report the mean milliseconds per launch
 * (CUDA events on the context stream) and algorithmic bytes per launch. */
ovl_status ovl_bench_wilson(ovl_ctx* ctx, int prec, int n, int iters, double* ms_per_launch,
                            double* bytes_per_launch);

/* FP32 instruction-issue probe: eight independent FMA chains per thread on every SM;
 * *fma_per_s receives the measured FP32 FMA instructions per second of this device (the
 * denominator of the ALU view of the double-float kernels, which run on the FP32 pipes).
 * Allocates and frees a small result buffer. */
ovl_status ovl_bench_fp32(ovl_ctx* ctx, double* fma_per_s);

/* Wilson-kernel autotuner result for one storage precision (OVL_PREC_*): the variant
 * in use (0 one thread per site, 1 one thread per site and direction, 2 4D tiles, 3 two
 * threads per site, one per half spinor, double-float only) and the measured
 * milliseconds per launch of each on this lattice (zero when the variant was forced, does
 * not apply to the precision or, for tiles, when the lattice does not divide into them).
 * Any output pointer may be NULL. */
ovl_status ovl_wilson_tuning(const ovl_ctx* ctx, int prec, int* variant, double* ms_thread_per_site,
                             double* ms_split, double* ms_tiled, double* ms_pair);

/* Library version string. */
const char* ovl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OVERLAP_H */
