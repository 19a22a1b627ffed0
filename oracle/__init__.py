"""Plain, slow FP64 CPU oracle for the overlap inverter of Cundy & Lee,
"The eigSUMR inverter for overlap fermions" (arXiv:1501.01855).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import or run anything in this package. The
product library never calls it, and this package never calls the product
library; the two share nothing but the seeded generators in ``synth``.

Each function states the passage of the paper it writes out. Everything works
in complex128 on the canonical layouts documented in ``synth``.

Modules
  wilson     gamma matrices, Wilson kernel K (Sec. 1, Eq. for aK_xy), dense K
  zolotarev  Zolotarev coefficients omega_i, sigma_i and Delta (Sec. 3)
  overlap    sign(K) (spectral definition, Sec. 1), epsilon(K) by per-pole CG,
             the sign with the smallest eigenvectors of K deflated (Sec. 1),
             D(mu), H = gamma5 D, D^dagger D (Sec. 1)
  solvers    Alg. 1 basis, minimal-residual (GMRES) iterates, GMRESR (Alg. 3),
             preconditioned CGNE (Alg. 4), dense solves
  eigen      Ritz recalculation (Alg. 6), eigSUMR subspace build (Alg. 5)
  deflation  Galerkin start, SUMR least-squares start, spectral preconditioner (Sec. 4)
  force      dS/dU for S = phi^dagger (D^dagger D)^-1 phi through the rational
             approximation (not in the paper; derivation in force.py)

Parity unpinned: none of the functions above is left without a pin; the pins
live in tests/test_oracle_*.py, and tests/test_oracle_planted_mistakes.py checks
that they fail when plausible mistakes are planted in these modules (one expression
of one function at a time).
"""
