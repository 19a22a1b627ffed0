"""Gauge-link gradient of S = phi^dag (D^dag D)^-1 phi through the Zolotarev
rational (the paper has no force; this is the derivative of the operator of
Secs. 1 and 3 with the coefficients omega_i, sigma_i held fixed).

Derivation. With H = gamma5 D = (1+mu)/2 gamma5 + (1-mu)/2 eps(K) (Hermitian),
D^dag D = H^2 (gamma5-hermiticity, Sec. 1). For chi = H^-2 phi and psi = H chi,

  dS = -chi^dag d(H^2) chi = -2 Re[psi^dag dH chi],  dH = (1-mu)/2 d eps(K),
  d eps(K) = sum_i omega_i [dK R_i - K R_i (dK K + K dK) R_i],  R_i = (K^2+sigma_i)^-1.

With a_i = R_i chi and b_i = R_i K psi:

  dS = -(1-mu) sum_i omega_i Re[ psi^dag dK a_i - b_i^dag dK (K a_i) - (K b_i)^dag dK a_i ].

For one link U_mu(s), Re[x^dag dK y] = -kappa Re sum_ab conj(dU_ab) (conj(F_ab) + G_ba) with
F_ab = sum conj(x(s)_{alpha a}) [g5 (1-g_mu)]_{alpha beta} y(s+mu)_{beta b} and
G_ab = sum conj(x(s+mu)_{alpha a}) [g5 (1+g_mu)]_{alpha beta} y(s)_{beta b}.
The returned gradient G_link (canonical link layout) is defined by
dS = 2 Re sum_links sum_ab conj(G_link_ab) dU_ab. Test infrastructure only.
"""
import numpy as np

from . import wilson, overlap


def link_outer(x, y, m0, antiperiodic_t=False):
    """Gradient array of Re[x^dag dK y] in the convention dX = 2 Re <G, dU>."""
    kap = wilson.kappa_of_m(m0)
    g5 = wilson.GAMMA5
    out = np.zeros(x.shape[:4] + (4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        P1 = g5 @ (wilson.I4 - wilson.GAMMA[mu])
        P2 = g5 @ (wilson.I4 + wilson.GAMMA[mu])
        yf = wilson.shift(y, mu, +1, antiperiodic_t)        # y(s+mu)
        xf = wilson.shift(x, mu, +1, antiperiodic_t)        # x(s+mu)
        F = np.einsum("...pa,pq,...qb->...ab", np.conj(x), P1, yf)
        G = np.einsum("...pa,pq,...qb->...ab", np.conj(xf), P2, y)
        out[..., mu, :, :] = -0.5 * kap * (np.conj(F) + np.swapaxes(G, -1, -2))
    return out


def apply_H(U, v, m0, mu, omega, sigma, tol, antiperiodic_t=False):
    return wilson.apply_gamma5(overlap.overlap_apply(U, v, m0, mu, omega, sigma, tol, antiperiodic_t))


def action(U, phi, m0, mu, omega, sigma, tol=1e-13, antiperiodic_t=False):
    """S = phi^dag (H^2)^-1 phi by CG on H^2 (returns (S, chi))."""
    H = lambda v: apply_H(U, v, m0, mu, omega, sigma, tol, antiperiodic_t)
    chi, _ = overlap.cg(lambda v: H(H(v)), phi, tol)
    return float(np.real(overlap.vdot(phi, chi))), chi


def gradient(U, phi, m0, mu, omega, sigma, tol=1e-13, antiperiodic_t=False):
    """G_link with dS = 2 Re sum conj(G) dU (canonical link layout)."""
    K = lambda v: wilson.apply_K(U, v, m0, antiperiodic_t)
    _, chi = action(U, phi, m0, mu, omega, sigma, tol, antiperiodic_t)
    psi = apply_H(U, chi, m0, mu, omega, sigma, tol, antiperiodic_t)
    Kpsi = K(psi)
    G = np.zeros(U.shape, dtype=np.complex128)
    for om, s in zip(omega, sigma):
        A = lambda v, s=s: K(K(v)) + s * v
        a, _ = overlap.cg(A, chi, tol)
        b, _ = overlap.cg(A, Kpsi, tol)
        Ka = K(a)
        Kb = K(b)
        c = -(1.0 - mu) * om
        G += c * (link_outer(psi, a, m0, antiperiodic_t)
                  - link_outer(b, Ka, m0, antiperiodic_t)
                  - link_outer(Kb, a, m0, antiperiodic_t))
    return G


def gradient_dense(U, phi, m0, mu, omega, sigma, antiperiodic_t=False):
    """The same gradient (same formula, same convention) with K as a dense matrix and the
    rational and shifted inverses from its eigendecomposition: for lattices up to 4^4,
    where the matrix-free CGs of gradient() take minutes. Returns (G, S)."""
    shape = phi.shape
    Kd = wilson.dense_K(U, m0, antiperiodic_t)
    lam, Q = np.linalg.eigh(Kd)
    Qh = np.conj(Q.T)
    eps = sum(om * lam / (lam * lam + s) for om, s in zip(omega, sigma))
    n = Kd.shape[0]
    G5 = overlap.gamma5_matrix(n // 12)
    H = 0.5 * (1.0 + mu) * G5 + 0.5 * (1.0 - mu) * (Q * eps) @ Qh
    H = 0.5 * (H + np.conj(H.T))
    f = phi.ravel()
    chi = np.linalg.solve(H @ H, f)
    S = float(np.real(np.vdot(f, chi)))
    psi = H @ chi
    Kpsi = Kd @ psi
    G = np.zeros(U.shape, dtype=np.complex128)
    for om, s in zip(omega, sigma):
        Ri = (Q * (1.0 / (lam * lam + s))) @ Qh
        a = Ri @ chi
        b = Ri @ Kpsi
        c = -(1.0 - mu) * om
        r = lambda v: v.reshape(shape)
        G += c * (link_outer(r(psi), r(a), m0, antiperiodic_t)
                  - link_outer(r(b), r(Kd @ a), m0, antiperiodic_t)
                  - link_outer(r(Kd @ b), r(a), m0, antiperiodic_t))
    return G, S
