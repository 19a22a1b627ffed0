"""Pins of the oracle's eigen accumulation (Sec. 5, Algs. 5-6) and deflation
(Sec. 4): Cholesky orthonormalisation equals Gram-Schmidt up to column phases;
Rayleigh-Ritz returns exact eigenpairs when they lie in the subspace and
otherwise interlaces; eigSUMR with the full Krylov space recovers the dense
spectrum; the Galerkin and least-squares starts satisfy their normal equations
and are exact for exact eigenvectors; the spectral preconditioner maps the
deflated eigenvalues of H^2 to c^2 = 3/4."""
import numpy as np

import synth
from oracle import overlap, eigen, deflation, wilson
from tests.oracle_util import dense_setup

DIMS = (2, 2, 2, 2)
NS = 16
MU = 0.05


def _ops():
    U, Kd, S, w = dense_setup(DIMS)
    D = overlap.dense_overlap(S, MU, NS)
    G5 = overlap.gamma5_matrix(NS)
    H = G5 @ D
    return D, H, G5, S


def test_cholesky_equals_gram_schmidt():
    rng = np.random.default_rng(0)
    V = rng.normal(size=(192, 10)) + 1j * rng.normal(size=(192, 10))
    E = V.conj().T @ V
    Uc = np.linalg.cholesky(E).conj().T
    Qc = V @ np.linalg.inv(Uc)
    Qg, _ = np.linalg.qr(V)
    ph = np.sum(Qg.conj() * Qc, axis=0)
    assert np.allclose(np.abs(ph), 1, atol=1e-12)
    assert np.allclose(Qc, Qg * ph, atol=1e-12)


def test_ritz_exact_in_subspace_and_interlacing():
    D, H, G5, S = _ops()
    delta = 0.01
    Mop = D.conj().T @ D + 2 * MU * delta * H
    lam_true, X = np.linalg.eigh(Mop)
    rng = np.random.default_rng(1)
    # subspace holding the 6 lowest exact eigenvectors plus 6 random vectors, mixed
    R = rng.normal(size=(192, 6)) + 1j * rng.normal(size=(192, 6))
    B = np.concatenate([X[:, :6], R], axis=1) @ (rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12)))
    VD = D @ B
    lam, Vn, VDn, res = eigen.ritz_recalculate(B, VD, MU, delta, 6, (NS, 4, 3))
    assert np.allclose(lam, lam_true[:6], atol=1e-10)
    # Ritz values of a random subspace interlace: lam_k(Ritz) >= lam_k(true)
    B2 = rng.normal(size=(192, 12)) + 1j * rng.normal(size=(192, 12))
    lam2, *_ = eigen.ritz_recalculate(B2, D @ B2, MU, delta, 12, (NS, 4, 3))
    assert np.all(lam2 >= lam_true[:12] - 1e-12)
    assert np.allclose(Vn.conj().T @ Vn, np.eye(6), atol=1e-10)


def test_eigsumr_equals_rayleigh_ritz_on_krylov_space():
    """Without a restart, Alg. 5 + Alg. 6 is Rayleigh-Ritz of D^dag D + 2 mu delta H
    over K_j(V, b); checked against an explicit QR-orthonormalised Krylov matrix,
    in the range of steps where the Alg. 1 basis is still orthonormal."""
    D, H, G5, S = _ops()
    V = G5 @ S
    b = synth.gaussian_source(DIMS, 5)
    delta = 0.01
    Mop = D.conj().T @ D + 2 * MU * delta * H
    j = 14
    lam, Vn, VDn, res = eigen.eigsumr_build(lambda q: (V @ q.ravel()).reshape(q.shape), b, MU, delta, 6, 400, j)
    Kr = np.stack([np.linalg.matrix_power(V, i) @ b.ravel() for i in range(j)], axis=1)
    Qk, _ = np.linalg.qr(Kr)
    ref = np.linalg.eigvalsh(Qk.conj().T @ Mop @ Qk)[:6]
    assert np.allclose(lam, ref, rtol=1e-9, atol=1e-12)
    # residuals recomputed from the dense operator: gamma5 D v - v (v, gamma5 D v)
    for i in range(6):
        v = Vn[:, i]
        r = H @ v - v * np.vdot(v, H @ v)
        assert np.isclose(res[i], np.linalg.norm(r), rtol=1e-8, atol=1e-12)
    # with restarts (m = 10, n = 4) the Ritz values still interlace the true ones
    lam2, *_ = eigen.eigsumr_build(lambda q: (V @ q.ravel()).reshape(q.shape), b, MU, delta, 4, 10, 18)
    lam_true = np.linalg.eigvalsh(Mop)
    assert np.all(lam2 >= lam_true[:4] - 1e-12)


def test_galerkin_and_ls_starts():
    D, H, G5, S = _ops()
    rng = np.random.default_rng(2)
    b = synth.gaussian_source(DIMS, 6)
    A = lambda v: (D @ v.ravel()).reshape(v.shape)
    Vr = [rng.normal(size=(NS, 4, 3)) + 1j * rng.normal(size=(NS, 4, 3)) for _ in range(5)]
    x0 = deflation.galerkin_start(A, Vr, b)
    Vm = np.stack([v.ravel() for v in Vr], axis=1)
    assert np.allclose(Vm.conj().T @ (b - A(x0)).ravel(), 0, atol=1e-11)
    # least-squares start: (D psi')^dag (b - D x0) = 0
    w, Y = np.linalg.eigh(H)
    psi = [Y[:, i].reshape(NS, 4, 3) for i in np.argsort(np.abs(w))[:8]]
    Dpsi = [A(p) for p in psi]
    x1 = deflation.sumr_ls_start(psi, Dpsi, b)
    DPm = np.stack([d.ravel() for d in Dpsi], axis=1)
    assert np.allclose(DPm.conj().T @ (b - A(x1)).ravel(), 0, atol=1e-11)
    # exact eigenvectors: x1 is the exact solution's component in their span
    xs = np.linalg.solve(D, b.ravel())
    P = np.stack([p.ravel() for p in psi], axis=1)
    assert np.allclose(P.conj().T @ x1.ravel(), P.conj().T @ xs, atol=1e-10)
    # with orthogonal D psi' the per-vector formula is the same minimiser
    x2 = deflation.sumr_ls_start(psi, Dpsi, b, per_vector=True)
    assert np.allclose(x1, x2, atol=1e-10)


def test_spectral_preconditioner_maps_to_c2():
    D, H, G5, S = _ops()
    w, Y = np.linalg.eigh(H)
    order = np.argsort(np.abs(w))
    idx = order[:10]
    psi = [Y[:, i].reshape(NS, 4, 3) for i in idx]
    mus = w[idx] ** 2
    P = deflation.spectral_precond(psi, mus)
    Pm = np.stack([P(e.reshape(NS, 4, 3)).ravel() for e in np.eye(192)], axis=1)
    M = Pm @ H @ H @ Pm
    for i in idx:
        assert np.isclose(np.vdot(Y[:, i], M @ Y[:, i]).real, 0.75, atol=1e-10)
    ev = np.linalg.eigvalsh(0.5 * (M + M.conj().T))
    assert np.sum(np.abs(ev - 0.75) < 1e-9) >= 10
