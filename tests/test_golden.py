"""Stored fixtures under tests/golden/ (written by tests/golden/make_golden.py from the
oracle alone): the oracle must keep reproducing them, the free-field spectrum is checked
against the dense operator, and the library's host-side Zolotarev coefficients and its GPU
overlap apply are compared with them (the GPU comparison needs no oracle at run time)."""
import os

import numpy as np
import pytest

import synth
from oracle import overlap, wilson, zolotarev

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#", ndmin=2)


def test_zolotarev_fixture_reproduced_by_oracle_and_library():
    g = load("zolotarev_n8_a0.15_b2.6.txt")
    om, sg, dl = zolotarev.zolotarev(8, 0.15, 2.6)
    order = np.argsort(sg)
    assert np.allclose(om[order], g[:-1, 0], rtol=1e-13, atol=0)
    assert np.allclose(sg[order], g[:-1, 1], rtol=1e-13, atol=0)
    # Delta is the maximum of |1 - eps(x)| found by a numerical search over [a, b], so it
    # is reproducible only to the search's resolution (platform libm differences)
    assert abs(dl - g[-1, 0]) <= 1e-6 * g[-1, 0]
    from paper_1501_01855_gb300 import binding as B
    lom, lsg, ldl = B.ovl_zolotarev_coeffs(8, 0.15, 2.6)
    o2 = np.argsort(lsg)
    assert np.allclose(lsg[o2], g[:-1, 1], rtol=1e-12, atol=0)
    assert np.allclose(lom[o2], g[:-1, 0], rtol=1e-12, atol=0)


def test_free_field_fixture_matches_dense_operator():
    g = load("free_field_absK_2x2x2x2_m1.4.txt")[:, 0]
    dims = (2, 2, 2, 2)
    Kd = wilson.dense_K(synth.unit_links(dims), 1.4)
    lam = np.sort(np.abs(np.linalg.eigvalsh(Kd)))
    assert np.allclose(lam, g, rtol=0, atol=1e-13)


def test_overlap_fixture_reproduced_by_oracle():
    g = load("overlap_exact_sign_2x2x2x2.txt")
    ref = g[:, 0] + 1j * g[:, 1]
    dims = (2, 2, 2, 2)
    U = synth.gauge_links(dims, 0.3, 1001)
    v = synth.gaussian_source(dims, 2001)
    S, _ = overlap.dense_sign(wilson.dense_K(U, 1.4))
    out = overlap.dense_overlap(S, 0.05, 16) @ v.ravel()
    assert np.linalg.norm(out - ref) <= 1e-14 * np.linalg.norm(ref)


@pytest.mark.gpu
def test_library_overlap_apply_matches_fixture():
    from tests.gpu_util import ctx
    g = load("overlap_exact_sign_2x2x2x2.txt")
    ref = (g[:, 0] + 1j * g[:, 1])
    dims = (2, 2, 2, 2)
    U = synth.gauge_links(dims, 0.3, 1001)
    v = synth.gaussian_source(dims, 2001)
    ev = np.abs(np.linalg.eigvalsh(wilson.dense_K(U, 1.4)))
    c = ctx(dims, U, mu=0.05, n_poles=24, eps=1e-12, a=0.95 * ev.min(), b=1.05 * ev.max())
    out = np.zeros_like(v)
    c.apply(v, out, eta=1e-12)
    assert np.linalg.norm(out.ravel() - ref) <= 1e-10 * np.linalg.norm(ref)
