"""Writes the stored expected values under tests/golden/ from the oracle alone.

    python tests/golden/make_golden.py

Every fixture records its inputs (seeds, sizes, parameters) in its header; the oracle
functions it calls and the passage they follow are named there too. Nothing here touches
the CUDA library.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import overlap, wilson, zolotarev  # noqa: E402

M0, MU = 1.4, 0.05


def write(name, header, rows):
    with open(os.path.join(HERE, name), "w") as f:
        for h in header:
            f.write("# " + h + "\n")
        for r in rows:
            f.write(" ".join("%.17e" % x for x in r) + "\n")


def main():
    # Zolotarev rational of Sec. 3 on [a, b] (oracle.zolotarev.zolotarev)
    n, a, b = 8, 0.15, 2.6
    om, sg, dl = zolotarev.zolotarev(n, a, b)
    write("zolotarev_n8_a0.15_b2.6.txt",
          ["Zolotarev coefficients, Sec. 3: eps(x) = sum_i omega_i x / (x^2 + sigma_i)",
           "n = 8, a = 0.15, b = 2.6; columns: omega_i sigma_i (ascending sigma); last row: Delta 0",
           "written by tests/golden/make_golden.py with oracle.zolotarev.zolotarev"],
          [(o, s) for o, s in sorted(zip(om, sg), key=lambda t: t[1])] + [(dl, 0.0)])
    # free-field |lambda(K)| on 2^4 in closed form (Sec. 1 operator at U = 1)
    dims = (2, 2, 2, 2)
    lam = np.sort(wilson.free_field_K_abs_spectrum(dims, M0))
    write("free_field_absK_2x2x2x2_m1.4.txt",
          ["|lambda(K)| of the free Wilson kernel K = gamma5 (1 - kappa hop), Sec. 1, U = 1",
           "lattice 2x2x2x2 periodic, m0 = 1.4; one value per row, ascending, with multiplicity",
           "written by tests/golden/make_golden.py with oracle.wilson.free_field_K_abs_spectrum (closed form)"],
          [(x,) for x in lam])
    # D(mu) v with the exact sign on a seeded 2^4 field (dense eigendecomposition)
    U = synth.gauge_links(dims, 0.3, 1001)
    v = synth.gaussian_source(dims, 2001)
    Kd = wilson.dense_K(U, M0)
    S, _ = overlap.dense_sign(Kd)
    D = overlap.dense_overlap(S, MU, 16)
    out = (D @ v.ravel()).reshape(v.shape)
    write("overlap_exact_sign_2x2x2x2.txt",
          ["D(mu) v, Sec. 1: D = 1/2 (1 + mu + (1 - mu) gamma5 sign(K)), exact sign by dense eigendecomposition",
           "lattice 2x2x2x2 periodic, m0 = 1.4, mu = 0.05; links synth.gauge_links(dims, 0.3, seed 1001),",
           "v = synth.gaussian_source(dims, seed 2001); rows in canonical order [t][z][y][x][spin][colour]: re im",
           "written by tests/golden/make_golden.py with oracle.wilson.dense_K, oracle.overlap.dense_sign, dense_overlap"],
          [(z.real, z.imag) for z in out.ravel()])


if __name__ == "__main__":
    main()
