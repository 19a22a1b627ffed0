"""Eigenvector accumulation of Sec. 5. Test infrastructure only.

* ritz_recalculate  Alg. 6: E_ij = (v_i, v_j); Cholesky E = U^dag U (L = U^dag);
                    M_ij = (v^D_i, v^D_j) + 2 mu delta (v_i, gamma5 v^D_j);
                    diagonalise L^-1 M U^-1 = Y Lambda Y^dag (ascending);
                    new v = V U^-1 Y, new v^D = V^D U^-1 Y (first n kept);
                    residuals r_i = gamma5 v^D_i - v_i (v_i, gamma5 v^D_i).
  Reading: the garbled "(V U^T v)" of Alg. 6 is the column combination
  V U^-1 Y, the only one that makes the kept vectors orthonormal Ritz vectors;
  the residual takes the gamma5 v^D form of Sec. 5.1.
* eigsumr_build     Alg. 5: the eigSUMR subspace build along the Alg. 1 basis,
                    v_k = q_j, v^D_k = (1-mu)/2 u + (1+mu)/2 q_j with u = U q_j,
                    recalculating at k == m and once at the end.
"""
import numpy as np

from .wilson import apply_gamma5


def _mat(vs):
    return np.stack([np.asarray(v).ravel() for v in vs], axis=1)


def ritz_recalculate(V, VD, mu, delta, n_keep, shape=None):
    """Alg. 6 on lists (or column matrices) of vectors. Returns
    (ritz_values[n_keep], Vnew (N x n_keep), VDnew (N x n_keep), residual norms)."""
    Vm = V if isinstance(V, np.ndarray) and V.ndim == 2 else _mat(V)
    VDm = VD if isinstance(VD, np.ndarray) and VD.ndim == 2 else _mat(VD)
    if shape is None:
        shape = (Vm.shape[0] // 12, 4, 3)
    E = np.conj(Vm.T) @ Vm
    Lc = np.linalg.cholesky(E)              # E = L L^dag, L lower
    Uc = np.conj(Lc.T)                      # E = U^dag U, U upper
    g5VD = np.stack([apply_gamma5(VDm[:, j].reshape(shape)).ravel()
                     for j in range(VDm.shape[1])], axis=1)
    M = np.conj(VDm.T) @ VDm + 2.0 * mu * delta * (np.conj(Vm.T) @ g5VD)
    Linv = np.linalg.inv(Lc)
    Uinv = np.linalg.inv(Uc)
    T = Linv @ M @ Uinv
    T = 0.5 * (T + np.conj(T.T))
    lam, Y = np.linalg.eigh(T)
    C = Uinv @ Y[:, :n_keep]
    Vn = Vm @ C
    VDn = VDm @ C
    res = []
    for i in range(n_keep):
        g5vd = apply_gamma5(VDn[:, i].reshape(shape)).ravel()
        r = g5vd - Vn[:, i] * np.vdot(Vn[:, i], g5vd)
        res.append(np.linalg.norm(r))
    return lam[:n_keep], Vn, VDn, np.array(res)


def eigsumr_build(applyU, b, mu, delta, n_keep, m_max, nsteps):
    """Alg. 5 for nsteps steps of Alg. 1. Returns (ritz values, V, VD, residuals)."""
    shape = b.shape
    q = b / np.linalg.norm(b.ravel())
    qt = q.copy()
    V, VD = [], []
    out = None
    for j in range(nsteps):
        u = applyU(q)
        V.append(q.ravel())
        VD.append((0.5 * (1 - mu) * u + 0.5 * (1 + mu) * q).ravel())
        if len(V) == m_max:
            lam, Vn, VDn, res = ritz_recalculate(V, VD, mu, delta, n_keep, shape)
            V = [Vn[:, i] for i in range(n_keep)]
            VD = [VDn[:, i] for i in range(n_keep)]
        g = -np.vdot(qt.ravel(), u.ravel())
        s = np.sqrt(1.0 - abs(g) ** 2)
        qn = (u + g * qt) / s
        qt = s * qt + np.conj(g) * qn
        q = qn
    return ritz_recalculate(V, VD, mu, delta, min(n_keep, len(V)), shape)
