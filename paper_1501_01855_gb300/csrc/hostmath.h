// Host FP64 numerics of liboverlap (no GPU): elliptic functions, Zolotarev
// coefficients, small dense complex linear algebra.
#pragma once
#include <complex>

namespace ovl {

// complete integral K(m) and sn, cn at parameter m; mc = 1 - m given separately
double ellip_K(double m, double mc);
void ellip_sncn(double u, double m, double mc, double* sn, double* cn);
// omega[n], sigma[n] (ascending sigma) and the maximum error delta; 0 on success
int zolotarev_coeffs(int n, double a, double b, double* omega, double* sigma, double* delta);
// max over a <= x <= b of x / (x^2 + sigma)
double pole_gbound(double sigma, double a, double b);

int cholesky_lower(int n, std::complex<double>* A);
void lower_inverse(int n, const std::complex<double>* L, std::complex<double>* Li);
void eigh_jacobi(int n, std::complex<double>* A, double* w, std::complex<double>* Z);
// Hermitian eigendecomposition (Householder tridiagonalisation + implicit QR; Jacobi as
// the fallback): w ascending, Z eigenvectors as columns, A destroyed
void eigh_herm(int n, std::complex<double>* A, double* w, std::complex<double>* Z);
int lu_solve(int n, std::complex<double>* A, std::complex<double>* B, int nb);
void tridiag_extremes(int n, const double* d, const double* e, double* lmin, double* lmax);

}  // namespace ovl
