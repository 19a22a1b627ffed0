// eigSUMR state (Sec. 5) shared by the accumulation hook and the C ABI.
#pragma once
#include <vector>

#include "context.h"
#include "solver.h"

namespace ovl {

struct EigState {
  int prec = P32;
  int m = 0, n_eig = 0, k = 0, n_seeded = 0;
  double mu = 0, delta = 0.01;
  double eps_v = 1e-4;      // desired eigenvector accuracy epsilon (Sec. 6 uses 1e-4)
  int kk = 25;              // iterations between accurate recalculations of v^D (Sec. 6: k = 25)
  int ndiag = 0;
  int cholesky_fallbacks = 0;
  double eta_cap = 1e-4;
  std::vector<double> uv_hist, ritz, res;
  Field* V = nullptr;
  Field* W = nullptr;
  EigHook* eig = nullptr;
  // eigCG: the previous step's t = Hhat^-1 p and z = H t of system 0
  Field* Tprev = nullptr;
  Field* Zprev = nullptr;
};

// the host part of a Ritz step (Alg. 6) on given Gram blocks (see eig.cu)
struct RitzHost {
  std::vector<double> lam, res;
  std::vector<std::complex<double>> C;   // k x keep, row-major
  int keep = 0;
  bool cholesky_fallback = false;
};
void ritz_host(int k, const std::complex<double>* E, const std::complex<double>* MVD, const std::complex<double>* G5,
               double mu, double delta, int keep, bool restart, RitzHost* out);

// keep the lowest `keep` Ritz vectors; restart = a basis restart inside the solve (also
// keeps the lowest Ritz vectors of the basis without its newest vector)
ovl_status ritz_step(ovl_ctx* c, EigState* e, int keep, bool restart = false);
ovl_status eig_hook(ovl_ctx* c, void* data, const Field& q, const Field& u, int iter);
ovl_status eig_cg_hook(ovl_ctx* c, void* data, const Field& t, const Field& z,
                       const std::vector<std::complex<double>>& beta_prev, const std::vector<double>& rnorm, int iter);

}  // namespace ovl
