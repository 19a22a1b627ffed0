"""Kernel low-mode deflation of the sign function (Sec. 1: the smallest eigenvectors of K
deflated, the Zolotarev rational covering the rest) through the C ABI, on 4^4 lattices
where the oracle has the dense spectrum: rough links (eps 0.7, smallest |lambda(K)| 0.036,
b/a = 70) and the benchmark's smooth ones (eps 0.3); and on 8^4 rough links against the
oracle's undeflated per-pole CG.

* the eigenvalues the library finds equal the dense ones of the oracle's K;
* the deflated sign (FP64 and double-float, multi-shift CG and stored-basis Lanczos)
  equals the oracle's spectral sign and the oracle's own deflated sign (its eigenvectors,
  its rational on its narrowed interval);
* deflation narrows the interval and the rational needs fewer poles and steps;
* n_ev = 0 restores the original rational (same result as before), and the fermion
  force refuses to run on a deflated context.
"""
import numpy as np
import pytest

import synth
from oracle import wilson, overlap, zolotarev as zo
from tests.gpu_util import lib, ctx, rel, M0

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


def _dense(eps, seed=1001):
    U = synth.gauge_links(DIMS, eps, seed)
    Kd = wilson.dense_K(U, M0)
    w, Q = np.linalg.eigh(Kd)
    S = (Q * np.sign(w)) @ np.conj(Q.T)
    return U, w, Q, S


@pytest.mark.parametrize("eps_links,n_ev", [(0.7, 10), (0.3, 6)])
def test_kernel_deflation_matches_spectral_sign(eps_links, n_ev):
    Bn = lib()
    U, w, Q, S = _dense(eps_links)
    order = np.argsort(np.abs(w))
    a, b = 0.95 * np.abs(w[order[0]]), 1.05 * np.max(np.abs(w))
    npoles = next(n for n in range(4, 40) if zo.zolotarev(n, a, b)[2] <= 1e-10)
    v = synth.gaussian_source(DIMS, 2101, nvec=2)
    exact = np.stack([(S @ x.ravel()).reshape(x.shape) for x in v])
    c = ctx(DIMS, U, a=a, b=b, n_poles=npoles, eps=1e-10, sign_method=1)
    before = np.zeros_like(v)
    c.sign_apply(v, before, eta=1e-11, prec=Bn.OVL_PREC_F64)
    lam, res, a_new, np_new, its = c.kernel_deflate(n_ev, tol=1e-11, max_iter=200)
    print("eps %.1f: %d eigenpairs in %d filter steps, max residual %.2e; a %.4f -> %.4f, poles %d -> %d"
          % (eps_links, n_ev, its, res.max(), a, a_new, npoles, np_new))
    assert np.all(res <= 1e-11)
    assert np.max(np.abs(np.sort(lam) - np.sort(w[order[:n_ev]]))) <= 1e-9
    assert a_new > a and np_new <= npoles
    # the oracle's own deflated sign: its eigenvectors, its rational on its narrowed interval
    psi = np.stack([Q[:, k].reshape(v[0].shape) for k in order[:n_ev]])
    a_or = 0.95 * np.abs(w[order[n_ev]])
    np_or = next(n for n in range(4, 40) if zo.zolotarev(n, a_or, b)[2] <= 1e-10)
    om, sg, _ = zo.zolotarev(np_or, a_or, b)
    oracle_defl = np.stack([overlap.deflated_sign_apply(U, x, M0, psi, w[order[:n_ev]], om, sg, tol=1e-14)
                            for x in v])
    for prec in (Bn.OVL_PREC_F64, Bn.OVL_PREC_F64E):
        for method in (0, 1):
            cm = ctx(DIMS, U, a=a, b=b, n_poles=npoles, eps=1e-10, sign_method=method)
            cm.kernel_deflate(n_ev, tol=1e-11, max_iter=200)
            out = np.zeros_like(v)
            cm.sign_apply(v, out, eta=1e-11, prec=prec)
            cm.close()
            e_s, e_o = rel(out, exact), rel(out, oracle_defl)
            print("  prec %d method %d: vs spectral sign %.2e, vs oracle deflated sign %.2e" % (prec, method, e_s, e_o))
            assert e_s <= 1e-9
            assert e_o <= 1e-9
    # undo: the original rational and the same result as before
    lam0, _, a0, np0, _ = c.kernel_deflate(0)
    assert np0 == npoles and abs(a0 - a) <= 1e-15 * a
    again = np.zeros_like(v)
    c.sign_apply(v, again, eta=1e-11, prec=Bn.OVL_PREC_F64)
    assert rel(again, before) <= 1e-13
    c.close()


def test_kernel_deflation_cuts_sign_steps_and_guards_the_force():
    """Rough links: the multi-shift CG of the deflated sign needs far fewer steps (the
    condition number of K^2 + sigma_0 falls with a^2), and overlap_force refuses to run
    until the deflation is removed."""
    Bn = lib()
    U, w, Q, S = _dense(0.7)
    a, b = 0.95 * np.min(np.abs(w)), 1.05 * np.max(np.abs(w))
    c = ctx(DIMS, U, a=a, b=b, n_poles=16, eps=1e-10, sign_method=1)
    v = synth.gaussian_source(DIMS, 2102)
    out = np.zeros_like(v)
    c.profile_reset()
    c.profile_enable(True)
    c.sign_apply(v, out, eta=1e-10, prec=Bn.OVL_PREC_F64)
    c.profile_enable(False)
    k_plain = c.profile_get()["wilson_f64"]["launches"]
    c.kernel_deflate(12, tol=1e-11, max_iter=200)
    c.profile_reset()
    c.profile_enable(True)
    c.sign_apply(v, out, eta=1e-10, prec=Bn.OVL_PREC_F64)
    c.profile_enable(False)
    k_defl = c.profile_get()["wilson_f64"]["launches"]
    print("Wilson launches per sign: %d undeflated, %d with 12 deflated modes" % (k_plain, k_defl))
    assert k_defl < 0.6 * k_plain
    assert rel(out, (S @ v.ravel()).reshape(v.shape)) <= 1e-9
    with pytest.raises(Bn.OvlError):
        c.force(v, tol=1e-10)
    c.kernel_deflate(0)
    G, _ = c.force(v, tol=1e-10)
    assert np.all(np.isfinite(G))
    c.close()


def test_kernel_deflation_8888_rough_links_matches_oracle():
    """8^4 rough links (eps 0.7; smallest |lambda(K)| 0.056): the overlap apply with 16
    eigenvectors of K deflated (double-float, stored-basis Lanczos, eta 1e-10) against the
    oracle's undeflated per-pole CG with its own Zolotarev rational on [0.05, 2.5] (both
    within 1e-10 of D with the exact sign), on two vectors, element by element."""
    import os
    Bn = lib()
    dims = (8, 8, 8, 8)
    a, b = 0.05, 2.5
    U = synth.gauge_links(dims, 0.7, 1006)
    v = synth.gaussian_source(dims, 2006, nvec=2)
    npoles = next(n for n in range(4, 40) if zo.zolotarev(n, a, b)[2] <= 1e-10)
    c = ctx(dims, U, a=a, b=b, n_poles=npoles, eps=1e-10, mu=0.05)
    lam, res, a_new, np_new, its = c.kernel_deflate(16, tol=1e-10, max_iter=400)
    out = np.zeros_like(v)
    c.apply(v, out, eta=1e-10, prec=Bn.OVL_PREC_F64E)
    c.close()
    om, sg, _ = zo.zolotarev(npoles, a, b)
    workers = max(1, min(16, len(os.sched_getaffinity(0))))
    ref = overlap.overlap_apply_many(U, v, M0, 0.05, om, sg, tol=1e-14, workers=workers)
    for j in range(2):
        err = rel(out[j], ref[j])
        pointwise = np.abs(out[j] - ref[j]).max() / np.abs(ref[j]).max()
        print("8^4 eps 0.7, 16 modes deflated (a %.4f -> %.4f, poles %d -> %d): vector %d relative %.2e, "
              "pointwise %.2e" % (a, a_new, npoles, np_new, j, err, pointwise))
        assert err <= 1e-9 and pointwise <= 1e-9
