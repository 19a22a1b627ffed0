"""Pins of the oracle's overlap operator (Sec. 1) and sign function (Secs. 1, 3):
sign(K)^2 = 1, the Zolotarev error bound against the spectral sign, per-pole CG
against the dense rational, the Ginsparg-Wilson relation, gamma5-hermiticity,
the circle spectrum, normality, [gamma5, D^dag D] = 0, the mass dependence of
D^dag D, and the free-field overlap spectrum in closed form."""
import numpy as np
import pytest

import synth
from oracle import wilson, overlap, zolotarev as zo
from tests.oracle_util import dense_setup

DIMS = (2, 2, 2, 2)
NS = 16


def test_sign_squares_to_one():
    U, Kd, S, w = dense_setup(DIMS)
    assert np.allclose(S @ S, np.eye(S.shape[0]), atol=1e-12)
    assert np.allclose(S, S.conj().T, atol=1e-13)


def test_zolotarev_bound_and_per_pole_cg():
    U, Kd, S, w = dense_setup(DIMS)
    a, b = 0.99 * np.min(np.abs(w)), 1.01 * np.max(np.abs(w))
    om, sg, delta = zo.zolotarev(6, a, b)
    E = overlap.dense_zolotarev_sign(Kd, om, sg)
    assert np.linalg.norm(E - S, 2) <= delta * (1 + 1e-8) + 1e-14
    v = synth.gaussian_source(DIMS, 4)
    got = overlap.zolotarev_sign_apply(U, v, 1.4, om, sg, tol=1e-14)
    ref = (E @ v.ravel()).reshape(v.shape)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


def _D(S, mu):
    return overlap.dense_overlap(S, mu, NS)


def test_ginsparg_wilson():
    _, _, S, _ = dense_setup(DIMS)
    D0 = _D(S, 0.0)
    G5 = overlap.gamma5_matrix(NS)
    gw = D0 @ G5 @ (np.eye(D0.shape[0]) - 2 * D0) + G5 @ D0
    assert np.max(np.abs(gw)) < 1e-12


@pytest.mark.parametrize("mu", [0.0, 0.05, 0.3])
def test_gamma5_hermiticity_circle_normality(mu):
    _, _, S, _ = dense_setup(DIMS)
    D = _D(S, mu)
    G5 = overlap.gamma5_matrix(NS)
    assert np.allclose(D.conj().T, G5 @ D @ G5, atol=1e-13)
    assert np.allclose(D @ D.conj().T, D.conj().T @ D, atol=1e-12)
    lam = np.linalg.eigvals(D)
    assert np.allclose(np.abs(lam - (1 + mu) / 2), (1 - mu) / 2, atol=1e-12)
    DD = D.conj().T @ D
    assert np.allclose(G5 @ DD, DD @ G5, atol=1e-12)
    D0 = _D(S, 0.0)
    assert np.allclose(DD, mu ** 2 * np.eye(DD.shape[0]) + (1 - mu ** 2) * D0.conj().T @ D0, atol=1e-12)


@pytest.mark.parametrize("dims,apt", [((2, 2, 2, 2), False), ((2, 2, 2, 4), True)])
def test_free_field_overlap_spectrum(dims, apt):
    mu = 0.05
    U = synth.unit_links(dims)
    Kd = wilson.dense_K(U, 1.4, apt)
    S, _ = overlap.dense_sign(Kd)
    ns = int(np.prod(dims))
    lam = np.linalg.eigvals(overlap.dense_overlap(S, mu, ns))
    ref = overlap.free_field_overlap_spectrum(dims, 1.4, mu, apt)
    key = lambda z: (np.round(z.real, 9), np.round(z.imag, 9))
    assert np.allclose(sorted(lam, key=key), sorted(ref, key=key), atol=1e-11)
    if not apt:
        # p = 0 gives lambda = mu, 12-fold (exact zero modes of D(0))
        assert np.sum(np.abs(lam - mu) < 1e-10) == 12


def test_matrix_free_overlap_matches_dense():
    U, Kd, S, w = dense_setup(DIMS)
    a, b = 0.99 * np.min(np.abs(w)), 1.01 * np.max(np.abs(w))
    om, sg, delta = zo.zolotarev(12, a, b)
    v = synth.gaussian_source(DIMS, 9)
    got = overlap.overlap_apply(U, v, 1.4, 0.05, om, sg, tol=1e-14)
    ref = (_D(S, 0.05) @ v.ravel()).reshape(v.shape)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
    gd = overlap.overlap_apply_dagger(U, v, 1.4, 0.05, om, sg, tol=1e-14)
    assert np.linalg.norm(gd - (_D(S, 0.05).conj().T @ v.ravel()).reshape(v.shape)) <= 1e-11 * np.linalg.norm(ref)


def test_pooled_per_pole_solves_match():
    """The batched form (every pole of every vector by its own CG, in a spawn-context
    process pool, sparse K) equals the single-vector per-pole CG on 4^4 and the dense
    Zolotarev rational evaluated on the spectrum of K on 2^4."""
    from oracle import zolotarev as zo
    dims = (4, 4, 4, 4)
    U = synth.gauge_links(dims, 0.3, 1001)
    om, sg, _ = zo.zolotarev(8, 0.2, 2.6)
    vs = synth.gaussian_source(dims, 5, nvec=2)
    out, its = overlap.zolotarev_sign_apply_many(U, vs, 1.4, om, sg, tol=1e-13, workers=2)
    for j in range(2):
        ref = overlap.zolotarev_sign_apply(U, vs[j], 1.4, om, sg, tol=1e-13)
        assert np.linalg.norm(out[j] - ref) <= 1e-11 * np.linalg.norm(ref)
    assert len(its) == 2 and len(its[0]) == 8
    d2 = (2, 2, 2, 2)
    U2, Kd, S, w = dense_setup(d2)
    v2 = synth.gaussian_source(d2, 6, nvec=2)
    R = overlap.dense_zolotarev_sign(Kd, om, sg)
    D = overlap.overlap_apply_many(U2, v2, 1.4, [0.05, 0.3], om, sg, tol=1e-14, workers=1)
    G5 = overlap.gamma5_matrix(16)
    for j, mu in enumerate((0.05, 0.3)):
        ref = 0.5 * (1 + mu) * v2[j].ravel() + 0.5 * (1 - mu) * (G5 @ (R @ v2[j].ravel()))
        assert np.linalg.norm(D[j].ravel() - ref) <= 1e-11 * np.linalg.norm(ref)


def test_deflated_sign_pins():
    """Sec. 1: sign(K) with the smallest eigenvectors of K deflated and the Zolotarev
    rational on the interval left over. With the exact low eigenvectors the result is
    within Delta(n, a', b) of the spectral sign, although the same rational without the
    deflation is far off (its interval no longer covers the low modes); no deflated vectors
    reduces to the plain rational; deflating every eigenvector gives the spectral sign."""
    U, Kd, S, w = dense_setup(DIMS)
    wv, Q = np.linalg.eigh(Kd)
    order = np.argsort(np.abs(wv))
    v = synth.gaussian_source(DIMS, 5)
    ref = (S @ v.ravel()).reshape(v.shape)
    nd = 12
    lam = wv[order[:nd]]
    psi = np.stack([Q[:, k].reshape(v.shape) for k in order[:nd]])
    a2 = 0.99 * np.abs(wv[order[nd]])
    b = 1.01 * np.max(np.abs(wv))
    om, sg, delta = zo.zolotarev(6, a2, b)
    got = overlap.deflated_sign_apply(U, v, 1.4, psi, lam, om, sg, tol=1e-14)
    err = np.linalg.norm(got - ref) / np.linalg.norm(v)
    plain = overlap.zolotarev_sign_apply(U, v, 1.4, om, sg, tol=1e-14)
    err_plain = np.linalg.norm(plain - ref) / np.linalg.norm(v)
    assert err <= delta * (1 + 1e-6) + 1e-12
    assert err_plain > 100 * delta
    # no deflated vectors: the plain rational
    none = overlap.deflated_sign_apply(U, v, 1.4, psi[:0], lam[:0], om, sg, tol=1e-14)
    assert np.linalg.norm(none - plain) <= 1e-13 * np.linalg.norm(plain)
    # every eigenvector deflated: the spectral sign exactly, whatever the rational
    allpsi = np.stack([Q[:, k].reshape(v.shape) for k in range(Q.shape[1])])
    full = overlap.deflated_sign_apply(U, v, 1.4, allpsi, wv, om, sg, tol=1e-14)
    assert np.linalg.norm(full - ref) <= 1e-11 * np.linalg.norm(ref)


def test_batched_forms_in_process_match_dense():
    """The batched per-pole forms run in this process (workers = 1): every (vector, pole)
    pair by its own CG, each vector's solutions summed with its own weights, then K and
    D(mu) per vector with its own mass, against the dense rational on 2^4."""
    from oracle import zolotarev as zo
    d2 = (2, 2, 2, 2)
    U2, Kd, S, w = dense_setup(d2)
    om, sg, _ = zo.zolotarev(6, 0.2, 2.6)
    vs = synth.gaussian_source(d2, 16, nvec=3)
    R = overlap.dense_zolotarev_sign(Kd, om, sg)
    G5 = overlap.gamma5_matrix(16)
    s, its = overlap.zolotarev_sign_apply_many(U2, vs, 1.4, om, sg, tol=1e-14, workers=1)
    mus = [0.05, 0.3, 0.6]
    D = overlap.overlap_apply_many(U2, vs, 1.4, mus, om, sg, tol=1e-14, workers=1)
    for j, mu in enumerate(mus):
        v = vs[j].ravel()
        assert np.linalg.norm(s[j].ravel() - R @ v) <= 1e-11 * np.linalg.norm(v)
        ref = 0.5 * (1 + mu) * v + 0.5 * (1 - mu) * (G5 @ (R @ v))
        assert np.linalg.norm(D[j].ravel() - ref) <= 1e-11 * np.linalg.norm(ref)
    assert len(its) == 3 and all(len(i) == 6 for i in its)
