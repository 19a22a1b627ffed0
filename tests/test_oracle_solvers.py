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


def _dense_H(mu=0.05):
    """H = gamma5 D(mu) on the 2^4 lattice with the exact sign (Sec. 1), dense."""
    from oracle import overlap
    from tests.oracle_util import dense_setup
    U, Kd, S, w = dense_setup((2, 2, 2, 2))
    D = overlap.dense_overlap(S, mu, 16)
    H = overlap.gamma5_matrix(16) @ D
    return 0.5 * (H + H.conj().T)


def test_cgne_spectral_with_exact_eigenvectors():
    """Alg. 4 with the spectral preconditioner of Sec. 4 built from the 12 lowest exact
    eigenvectors of H^2 (H = gamma5 D, 2^4): the solution solves H x = b, the CG iterates
    are those of plain CG on the explicit matrix Hhat^-1 H^2 Hhat^-1 (one-sided use of
    Hhat^-1, or a wrong final x = H Hhat^-1 x_j, would break one of the two), the
    preconditioned operator has the deflated eigenvalues at c^2 = 3/4, and the solve takes
    fewer iterations than without the preconditioner."""
    from oracle import deflation
    H = _dense_H()
    lam, Q = np.linalg.eigh(H @ H)
    n = 12
    shape = (16, 4, 3)
    psi = [Q[:, i].reshape(shape) for i in range(n)]
    pre = deflation.spectral_precond(psi, lam[:n])
    rng = np.random.default_rng(5)
    b = (rng.normal(size=shape) + 1j * rng.normal(size=shape))
    applyH = lambda v: (H @ v.ravel()).reshape(v.shape)
    x, it = solvers.cgne_spectral(applyH, b, 1e-12, pre)
    assert np.linalg.norm(applyH(x) - b) <= 1e-10 * np.linalg.norm(b)
    assert np.allclose(x.ravel(), np.linalg.solve(H, b.ravel()), rtol=0, atol=1e-9 * np.linalg.norm(x))
    # the explicit preconditioned operator: deflated eigenvalues at c^2 = 3/4, others kept
    P = np.stack([pre(np.eye(192)[:, j].reshape(shape)).ravel() for j in range(192)], axis=1)
    M = P @ H @ H @ P
    for i in range(n):
        assert np.allclose(M @ Q[:, i], 0.75 * Q[:, i], atol=1e-10)
    for i in range(n, n + 5):
        assert np.allclose(M @ Q[:, i], lam[i] * Q[:, i], atol=1e-10)
    # plain CG on M with rhs Hhat^-1 b gives the same solution through x = H Hhat^-1 y
    y = np.linalg.solve(M, P @ b.ravel())
    assert np.allclose(x.ravel(), H @ (P @ y), atol=1e-9 * np.linalg.norm(x))
    _, it0 = solvers.cgne_spectral(applyH, b, 1e-12, lambda v: v)
    assert it < it0, (it, it0)


def test_gmres_solve_matches_dense_solve():
    """The restarted minimal-residual solve reaches ||b - A x|| <= tol ||b|| and the
    dense solution, with restarts (restart length 15 < the 60 steps needed)."""
    U, rho, b = _shifted_unitary(N=100, mu=0.02, seed=8)
    A = rho * np.eye(len(b)) + U
    x = solvers.gmres_solve(lambda v: A @ v, b, 1e-12, restart=15)
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
