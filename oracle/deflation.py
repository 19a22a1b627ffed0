"""Deflation of the middle solve, Sec. 4. Test infrastructure only.

* galerkin_start      x0 = x~0 + V (V^dag A V)^-1 V^dag (b - A x~0).
* sumr_ls_start       rotate psi' = psi Y so that (psi'_i, gamma5 D psi'_j) is
                      diagonal, then choose alpha to minimise ||b - sum_j alpha_j D psi'_j||;
                      x0 = sum_j alpha_j psi'_j. The printed per-vector formula
                      alpha_j = (D psi'_j, b)/(D psi'_j, D psi'_j) is the minimiser
                      only when the D psi'_j are mutually orthogonal; the general
                      minimiser (least-squares normal equations) is used, and the
                      per-vector form is kept behind a flag.
* spectral_precond    Hhat^-1 = 1 + sum_i psi_i psi_i^dag (c / sqrt(mu_i) - 1), c = sqrt(3)/2.
"""
import numpy as np

from .wilson import apply_gamma5


def _cols(vs):
    return np.stack([np.asarray(v).ravel() for v in vs], axis=1)


def galerkin_start(applyA, V, b, x0t=None):
    Vm = _cols(V)
    shape = b.shape
    x0t = np.zeros_like(b) if x0t is None else x0t
    AV = np.stack([applyA(Vm[:, j].reshape(shape)).ravel() for j in range(Vm.shape[1])], axis=1)
    G = np.conj(Vm.T) @ AV
    r = (b - applyA(x0t)).ravel()
    y = np.linalg.solve(G, np.conj(Vm.T) @ r)
    return x0t + (Vm @ y).reshape(shape)


def sumr_ls_start(V, DV, b, per_vector=False):
    """V: approximate eigenvectors psi_i of gamma5 D (orthonormal columns); DV = D psi_i.
    Returns x0 (shape of b)."""
    Vm = _cols(V)
    DVm = _cols(DV)
    shape = b.shape
    g5DV = np.stack([apply_gamma5(DVm[:, j].reshape(shape)).ravel() for j in range(DVm.shape[1])], axis=1)
    Hs = np.conj(Vm.T) @ g5DV
    Hs = 0.5 * (Hs + np.conj(Hs.T))
    _, Y = np.linalg.eigh(Hs)
    P = Vm @ Y
    DP = DVm @ Y
    bb = b.ravel()
    if per_vector:
        alpha = np.array([np.vdot(DP[:, j], bb) / np.vdot(DP[:, j], DP[:, j]) for j in range(DP.shape[1])])
    else:
        G = np.conj(DP.T) @ DP
        alpha = np.linalg.solve(G, np.conj(DP.T) @ bb)
    return (P @ alpha).reshape(shape)


def spectral_precond(V, mus, c=np.sqrt(3.0) / 2.0):
    """Return apply(x) = x + sum_i psi_i (psi_i, x) (c/sqrt(mu_i) - 1)."""
    Vm = _cols(V)
    f = c / np.sqrt(np.asarray(mus, dtype=np.float64)) - 1.0

    def apply(x):
        xs = x.ravel()
        return (xs + Vm @ (f * (np.conj(Vm.T) @ xs))).reshape(x.shape)
    return apply
