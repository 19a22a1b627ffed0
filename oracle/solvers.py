"""Solvers of Secs. 2-4, written from their definitions. Test infrastructure only.

* sumr_basis      Alg. 1: the short-recurrence orthonormal Krylov basis of a
                  unitary U (q, q-tilde, gamma_j, sigma_j).
* minres_iterates SUMR's iterates: for A = rho + U the SUMR iterate x_j is the
                  minimal-residual (GMRES) iterate over x0 + K_j(A, r0) (Sec. 2:
                  an efficient representation of GMRES). Written as Arnoldi with
                  twice-iterated Gram-Schmidt and a dense least-squares solve.
* gmresr          Alg. 3 with a caller-supplied preconditioner solve and product.
* cgne_spectral   Alg. 4: CG on Hhat^-1 H^2 Hhat^-1, x = H Hhat^-1 x_j.
"""
import numpy as np


def vdot(a, b):
    return np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel())


def norm(a):
    return float(np.sqrt(np.real(vdot(a, a))))


def sumr_basis(applyU, b, nsteps):
    """Alg. 1. Returns (Q list of q_0..q_nsteps, gamma[nsteps], sigma[nsteps])."""
    q = b / norm(b)
    qt = q.copy()
    Q = [q]
    gam = []
    sig = []
    for _ in range(nsteps):
        u = applyU(q)
        g = -vdot(qt, u)
        s = np.sqrt(1.0 - abs(g) ** 2)
        qn = (u + g * qt) / s
        qt = s * qt + np.conj(g) * qn
        q = qn
        Q.append(q)
        gam.append(g)
        sig.append(s)
    return Q, np.array(gam), np.array(sig)


def minres_iterates(applyA, b, nsteps, x0=None, callback=None):
    """Minimal-residual iterates x_j = argmin_{x in x0 + K_j(A, r0)} ||b - A x||.

    Returns (x_final, [||b - A x_j|| for j = 1..nsteps]) with true residuals.
    Stops early on an exact (lucky) breakdown.
    """
    x0 = np.zeros_like(b) if x0 is None else x0
    r0 = b - applyA(x0)
    beta = norm(r0)
    V = [r0 / beta]
    H = np.zeros((nsteps + 1, nsteps), dtype=np.complex128)
    hist = []
    x = x0
    for j in range(nsteps):
        w = applyA(V[j])
        for _ in range(2):
            for i in range(j + 1):
                h = vdot(V[i], w)
                H[i, j] += h
                w = w - h * V[i]
        H[j + 1, j] = norm(w)
        e1 = np.zeros(j + 2, dtype=np.complex128)
        e1[0] = beta
        y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
        x = x0 + sum(yi * vi for yi, vi in zip(y, V[:j + 1]))
        hist.append(norm(b - applyA(x)))
        if callback is not None:
            callback(j, x)
        if H[j + 1, j].real < 1e-300:
            break
        V.append(w / H[j + 1, j])
    return x, np.array(hist)


def gmres_solve(applyA, b, tol, restart=60, maxiter=10000):
    """Restarted minimal-residual solve to ||b - A x|| <= tol ||b|| (unrelaxed)."""
    x = np.zeros_like(b)
    nb = norm(b)
    it = 0
    while it < maxiter:
        r = b - applyA(x)
        if norm(r) <= tol * nb:
            break
        dx, hist = minres_iterates(applyA, r, restart)
        x = x + dx
        it += len(hist)
    return x


def gmresr(applyA, b, eps, precond_solve, product, maxouter=50):
    """Alg. 3 (GMRESR): x=0, r=b; while ||r|| > eps ||b||: u ~ A^-1 r,
    c ~ A u, orthogonalise c against the stored C (same combination on u),
    normalise by ||c||, alpha = (c, r), x += alpha u, r -= alpha c.

    precond_solve(r) -> u; product(u, r) -> c. Reading of the normalisation:
    nu = ||c|| is taken once, then c /= nu and u /= nu.
    Returns (x, list of ||r|| after each outer step).
    """
    x = np.zeros_like(b)
    r = b.copy()
    C, Us = [], []
    nb = norm(b)
    hist = []
    while norm(r) > eps * nb and len(C) < maxouter:
        u = precond_solve(r)
        c = product(u, r)
        for cj, uj in zip(C, Us):
            beta = vdot(cj, c)
            c = c - beta * cj
            u = u - beta * uj
        nu = norm(c)
        c = c / nu
        u = u / nu
        C.append(c)
        Us.append(u)
        alpha = vdot(c, r)
        x = x + alpha * u
        r = r - alpha * c
        hist.append(norm(r))
    return x, hist


def cgne_spectral(applyH, b, eps, apply_Hhat_inv, maxiter=100000):
    """Alg. 4: preconditioned CGNE for H x = b with Hermitian H and a Hermitian
    preconditioner Hhat^-1 used on both sides of H^2.
      r0 = p0 = Hhat^-1 b; loop z = Hhat^-1 H^2 Hhat^-1 p, ...; x = H Hhat^-1 x_j.
    Returns (x, iterations).
    """
    r = apply_Hhat_inv(b)
    p = r.copy()
    x = np.zeros_like(b)
    rr = np.real(vdot(r, r))
    nb = norm(b)
    j = 0
    while np.sqrt(rr) >= nb * eps and j < maxiter:
        z = apply_Hhat_inv(applyH(applyH(apply_Hhat_inv(p))))
        alpha = rr / vdot(r, z)
        r = r - alpha * z
        x = x + alpha * p
        rr_new = np.real(vdot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        j += 1
    return applyH(apply_Hhat_inv(x)), j
