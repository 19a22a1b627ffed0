"""Pins of the oracle's solvers (Secs. 2-4): Alg. 1 gives an orthonormal basis
with a unitary upper-Hessenberg projection; the minimal-residual iterates equal a
brute-force least-squares over an explicit Krylov matrix; GMRESR (Alg. 3)
converges in one step with an exact inner solve and never increases the
residual; preconditioned CGNE (Alg. 4) solves H x = b."""
import numpy as np
import pytest

from oracle import solvers


def _shifted_unitary(N=120, mu=0.05, seed=3):
    rng = np.random.default_rng(seed)
    Z = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    Q, R = np.linalg.qr(Z)
    U = Q * (np.diag(R) / np.abs(np.diag(R)))
    rho = (1 + mu) / (1 - mu)
    b = rng.normal(size=N) + 1j * rng.normal(size=N)
    return U, rho, b


def test_alg1_basis():
    U, rho, b = _shifted_unitary()
    Q, gam, sig = solvers.sumr_basis(lambda v: U @ v, b, 30)
    Qm = np.stack(Q[:30], axis=1)
    assert np.allclose(Qm.conj().T @ Qm, np.eye(30), atol=1e-10)
    B = Qm.conj().T @ U @ Qm
    assert np.allclose(np.tril(B, -2), 0, atol=1e-10)
    # B is the leading block of a unitary Hessenberg matrix: columns 0..28 are orthonormal
    # once the subdiagonal row 30 (sigma_29) is appended
    Bfull = np.stack(Q[:31], axis=1).conj().T @ U @ Qm
    assert np.allclose(Bfull.conj().T @ Bfull, np.eye(30), atol=1e-10)
    assert np.allclose(np.diag(Bfull, -1), sig, atol=1e-10)
    # the first column of B is (-gamma_0, sigma_0)
    assert np.isclose(Bfull[0, 0], -gam[0]) and np.isclose(Bfull[1, 0], sig[0])


def test_minres_iterates_brute_force():
    U, rho, b = _shifted_unitary(N=60)
    A = rho * np.eye(60) + U
    x, hist = solvers.minres_iterates(lambda v: A @ v, b, 12)
    for j in range(1, 13):
        Kr = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(j)], axis=1)
        y = np.linalg.lstsq(A @ Kr, b, rcond=None)[0]
        assert np.isclose(hist[j - 1], np.linalg.norm(b - A @ Kr @ y), rtol=1e-8)
    assert np.all(np.diff(hist) <= 1e-12)
    x60, h60 = solvers.minres_iterates(lambda v: A @ v, b, 60)
    assert np.allclose(x60, np.linalg.solve(A, b), atol=1e-10)


def test_gmresr_exact_inner_one_step():
    U, rho, b = _shifted_unitary()
    A = rho * np.eye(len(b)) + U
    x, hist = solvers.gmresr(lambda v: A @ v, b, 1e-12,
                             lambda r: np.linalg.solve(A, r), lambda u, r: A @ u)
    assert len(hist) == 1
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b)


def test_gmresr_inexact_inner_monotone():
    U, rho, b = _shifted_unitary()
    A = rho * np.eye(len(b)) + U
    rng = np.random.default_rng(1)

    def inner(r):
        u = np.linalg.solve(A, r)
        return u + 1e-2 * np.linalg.norm(u) * (rng.normal(size=u.shape) + 1j * rng.normal(size=u.shape)) / np.sqrt(2 * len(u))

    x, hist = solvers.gmresr(lambda v: A @ v, b, 1e-12, inner, lambda u, r: A @ u)
    assert np.all(np.diff(hist) <= 1e-14 * np.linalg.norm(b))
    assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
    assert len(hist) <= 8


def test_cgne_spectral_identity_precond():
    rng = np.random.default_rng(2)
    N = 80
    Z = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    H = Z + Z.conj().T + 0.5 * np.eye(N)
    b = rng.normal(size=N) + 1j * rng.normal(size=N)
    x, it = solvers.cgne_spectral(lambda v: H @ v, b, 1e-12, lambda v: v)
    assert np.linalg.norm(H @ x - b) <= 1e-9 * np.linalg.norm(b)
