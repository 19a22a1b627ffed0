// Solver entry points used by the C ABI (see solver.cu).
#pragma once
#include <vector>

#include "context.h"

namespace ovl {

// Called after every sign application of the middle SUMR solve (eigSUMR, Alg. 5):
// q holds q_j, u holds V q_j for every system of the batch.
typedef ovl_status (*SumrHook)(ovl_ctx* c, void* data, const Field& q, const Field& u, int iter);
typedef ovl_status (*OuterHook)(ovl_ctx* c, void* data, int outer);
// Called in every step j of the middle relCG solve (eigCG, Sec. 5) once z_j = H t_j is
// known, t_j = Hhat^-1 p_j: with beta_{j-1} (the previous step's beta, 0 at j = 0) and
// ||r_j||, both per system, the residual direction Hhat^-1 r_j = t_j - beta_{j-1} t_{j-1}
// and D Hhat^-1 r_j = gamma5 (z_j - beta_{j-1} z_{j-1}) follow from vectors CG computes.
typedef ovl_status (*CgHook)(ovl_ctx* c, void* data, const Field& t, const Field& z,
                             const std::vector<std::complex<double>>& beta_prev,
                             const std::vector<double>& rnorm, int iter);

// State of the SUMR short recurrence of one system (see sumr_rec_step in solver.cu)
struct SumrRec {
  cd gprev = 0, sprev = 0;
  double cprev = 1, sigprev = 0;
  cd zeta = 1.0;
  cd ghat;   // residual estimate (complex; its modulus is ||r_j||)
  int it = 0;
};
ovl_status defl_start_host(int n, const cd* VV, const cd* WW, const cd* WV, const cd* G5VV, const cd* G5VW,
                           int nsys, const cd* VB, const cd* WB, const double* mus, bool per_vector, cd* coefs);
bool sumr_basis_step(cd qtu, double uu, double tt, cd* gam, double* sig);
void sumr_rec_step(SumrRec& s, double rho, cd gam, double sig, cd vals[6]);

struct SumrCfg {
  int prec = P64;          // precision of the middle-solve vectors
  double target = 1e-3;    // relative residual target
  double relax = 1.0;      // relaxation factor
  double floor = 1e-2;     // sign accuracy never worse than this
  double eta_cap = 0.0;    // >0: sign accuracy never worse than this either (eigen accumulation)
  int maxit = 1000;
  int mode = -1;           // sign precision, -1: chosen by eta
  double qdrift = 0.1;     // stop when | ||q|| - 1 | exceeds this
  double eta_fixed = 0.0;  // >0: apply the sign at this accuracy every iteration (no relaxation)
  const double* eta_dyn = nullptr;   // set: the sign accuracy is *eta_dyn, read every iteration
  std::vector<double>* hist = nullptr;   // residual estimates ||r_j|| / ||b||, appended per iteration
  ovl_defl* defl = nullptr;
  SumrHook hook = nullptr;
  CgHook cg_hook = nullptr;
  void* hook_data = nullptr;
};

struct SumrResult {
  std::vector<int> iters;
  std::vector<double> resid;
  std::vector<long long> wcalls;
  std::vector<int> sign_calls;
  std::vector<int> stopped;   // 0 normal, 1 q drift, 2 breakdown
};

struct EigHook {
  bool active = false;
  double target = 1e-2;    // middle-solve target while accumulating (GMRESR converges in two steps)
  double eta_cap = 1e-4;   // sign accuracy during accumulation
  SumrHook hook = nullptr;
  CgHook cg_hook = nullptr;
  OuterHook after_outer = nullptr;
  void* data = nullptr;
};

ovl_status sumr_batch(ovl_ctx* c, const SumrCfg& cfg, int n, const std::vector<double>& mus, const Field& b, int boff,
                      Field& x, int xoff, SumrResult& res);
ovl_status cg_batch(ovl_ctx* c, const SumrCfg& cfg, int n, const std::vector<double>& mus, const Field& b, int boff,
                    Field& x, int xoff, SumrResult& res);
// nsrc > 0: the batch is every mass of nsrc sources, system q = mass * nsrc + source; the
// first middle solve (r = b) then shares one SUMR basis per source (sumr_multimass)
ovl_status gmresr_batch(ovl_ctx* c, int n, const std::vector<double>& mus, const Field& b, int boff, Field& x, int xoff,
                        double tol, ovl_defl* defl, ovl_solve_info* info, EigHook* eig, int nsrc = 0);
ovl_status sumr_multimass(ovl_ctx* c, const SumrCfg& cfg, int ns, int nm, const std::vector<double>& mus_m,
                          const Field& b, int boff, Field& x, int xoff, SumrResult& res);
ovl_status overlap_apply_batch(ovl_ctx* c, const Field& v, int voff, Field& out, int ooff, int n,
                               const std::vector<double>& mus, const std::vector<double>& eta, int herm, int mode,
                               long long* wcalls_out);
ovl_status dots_batch(ovl_ctx* c, const Field& x, int xoff, const Field& y, int yoff, int n, std::vector<cd>& out);
ovl_status norms_batch(ovl_ctx* c, const Field& x, int xoff, int n, std::vector<double>& out);
ovl_status axpby_batch(ovl_ctx* c, const std::vector<cd>& a, const Field& x, int xoff, const std::vector<cd>& b,
                       const Field& y, int yoff, Field& z, int zoff, int n);
ovl_status copy_convert(ovl_ctx* c, const Field& in, int ioff, Field& out, int ooff, int n);
ovl_status gram_device(ovl_ctx* c, const Field& A, int aoff, int na, const Field& B, int boff, int nb, int g5,
                       double** dG, int** derr);
ovl_status gram_host(ovl_ctx* c, const Field& A, int aoff, int na, const Field& B, int boff, int nb, int g5,
                     std::vector<cd>& G);
ovl_status combine_host(ovl_ctx* c, const Field& A, int aoff, int na, const std::vector<cd>& C, Field& Y, int yoff,
                        int ny, int add);
ovl_status defl_prepare(ovl_ctx* c, ovl_defl* d);

}  // namespace ovl
