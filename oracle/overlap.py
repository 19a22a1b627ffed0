"""Overlap operator (Sec. 1):

  D(mu) = 1/2 (1 + mu + (1 - mu) gamma5 sign(K)),

sign(K) either from its spectral definition (Sec. 1: sum_i psi_i psi_i^dag
sign(lambda_i) over the eigenpairs of the Hermitian K; dense eigh, small
lattices only) or from the Zolotarev rational of Sec. 3,

  epsilon(K) v = sum_i omega_i K (K^2 + sigma_i)^-1 v,

each shifted system solved by its own plain conjugate gradient (no multi-shift,
no pole dropping), optionally with the lowest eigenvectors of K taken out and
their sign applied exactly (Sec. 1: deflation of the smallest eigenvectors of K,
the approximation covering the rest of the spectrum). Test infrastructure only.
"""
import numpy as np

from . import wilson


# ---------------------------------------------------------------- dense forms
def dense_sign(Kd):
    """sign(K) = Q sign(Lambda) Q^dag for Hermitian dense K (Sec. 1)."""
    w, Q = np.linalg.eigh(Kd)
    return (Q * np.sign(w)) @ np.conj(Q.T), w


def dense_zolotarev_sign(Kd, omega, sigma):
    """epsilon(K) evaluated on the spectrum of dense Hermitian K."""
    w, Q = np.linalg.eigh(Kd)
    ew = sum(om * w / (w * w + s) for om, s in zip(omega, sigma))
    return (Q * ew) @ np.conj(Q.T)


def gamma5_matrix(nsites):
    g5 = np.diag(np.real(np.diag(wilson.GAMMA5)))
    return np.kron(np.eye(nsites), np.kron(g5, np.eye(3))).astype(np.complex128)


def dense_overlap(Sd, mu, nsites):
    """D(mu) = 1/2 (1 + mu + (1 - mu) gamma5 S) as a dense matrix."""
    n = Sd.shape[0]
    G5 = gamma5_matrix(nsites)
    return 0.5 * (1.0 + mu) * np.eye(n) + 0.5 * (1.0 - mu) * (G5 @ Sd)


# ---------------------------------------------------------------- matrix free
def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def norm(a):
    return float(np.sqrt(np.real(vdot(a, a))))


def cg(apply, b, tol, maxiter=100000):
    """Plain conjugate gradient for Hermitian positive definite apply(); stops at
    ||r|| <= tol * ||b||. Returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.real(vdot(r, r))
    stop = (tol * norm(b)) ** 2
    it = 0
    while rr > stop and it < maxiter:
        Ap = apply(p)
        alpha = rr / np.real(vdot(p, Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.real(vdot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


# ---------------------------------------------------------------- larger lattices
# The per-pole CGs of every (vector, pole) pair are independent, so they run in a pool of
# worker processes (spawn start method: the workers import only numpy, scipy and this
# package), each holding K as a sparse matrix (wilson.sparse_K).
_WORKER_K = None


def _worker_init(U, m0, antiperiodic_t):
    global _WORKER_K
    _WORKER_K = wilson.sparse_K(U, m0, antiperiodic_t)


def _worker_pole_solve(task):
    v, s, tol = task
    K = _WORKER_K
    return cg(lambda p: K @ (K @ p) + s * p, v, tol)


def shifted_solves(U, vs, m0, sigma, tol=1e-13, antiperiodic_t=False, workers=1):
    """x_ij = (K^2 + sigma_i)^-1 v_j by plain CG for every pole i and vector j (flat
    vectors), returned as xs[j][i] with the iteration counts its[j][i]. workers > 1 runs
    the solves in a spawn-context process pool; workers = 1 runs them here."""
    vs = np.asarray(vs)
    nv = vs.shape[0]
    tasks = [(vs[j].ravel(), float(s), tol) for j in range(nv) for s in sigma]
    if workers <= 1:
        _worker_init(U, m0, antiperiodic_t)
        res = [_worker_pole_solve(t) for t in tasks]
    else:
        import multiprocessing as mp
        import os
        # one BLAS thread per worker: the parallelism is the pool's
        keep = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in keep:
            os.environ[k] = "1"
        try:
            with mp.get_context("spawn").Pool(workers, initializer=_worker_init,
                                              initargs=(U, m0, antiperiodic_t)) as pool:
                res = pool.map(_worker_pole_solve, tasks, chunksize=1)
        finally:
            for k, v in keep.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    npol = len(sigma)
    xs = [[res[j * npol + i][0] for i in range(npol)] for j in range(nv)]
    its = [[res[j * npol + i][1] for i in range(npol)] for j in range(nv)]
    return xs, its


def zolotarev_sign_apply_many(U, vs, m0, omega, sigma, tol=1e-13, antiperiodic_t=False, workers=1):
    """epsilon(K) v_j = K sum_i omega_i (K^2 + sigma_i)^-1 v_j for a batch vs (n, ...),
    every pole of every vector by its own CG (shifted_solves). Returns (out, iterations)."""
    vs = np.asarray(vs)
    xs, its = shifted_solves(U, vs, m0, sigma, tol, antiperiodic_t, workers)
    K = wilson.sparse_K(U, m0, antiperiodic_t)
    out = np.empty_like(vs)
    for j in range(vs.shape[0]):
        y = sum(om * x for om, x in zip(omega, xs[j]))
        out[j] = (K @ y).reshape(vs.shape[1:])
    return out, its


def overlap_apply_many(U, vs, m0, mu, omega, sigma, tol=1e-13, antiperiodic_t=False, workers=1):
    """D(mu) v = 1/2 (1+mu) v + 1/2 (1-mu) gamma5 epsilon(K) v for a batch vs (n, ...);
    mu may be one mass or one per vector."""
    vs = np.asarray(vs)
    s, _ = zolotarev_sign_apply_many(U, vs, m0, omega, sigma, tol, antiperiodic_t, workers)
    mus = np.broadcast_to(np.asarray(mu, dtype=np.float64), (vs.shape[0],))
    out = np.empty_like(vs)
    for j in range(vs.shape[0]):
        out[j] = 0.5 * (1.0 + mus[j]) * vs[j] + 0.5 * (1.0 - mus[j]) * wilson.apply_gamma5(s[j])
    return out


def zolotarev_sign_apply(U, v, m0, omega, sigma, tol=1e-13, antiperiodic_t=False,
                         return_solutions=False):
    """epsilon(K) v = K sum_i omega_i (K^2 + sigma_i)^-1 v, every pole by its own CG."""
    K = lambda x: wilson.apply_K(U, x, m0, antiperiodic_t)
    y = np.zeros_like(v)
    sols = []
    for om, s in zip(omega, sigma):
        xi, _ = cg(lambda p, s=s: K(K(p)) + s * p, v, tol)
        sols.append(xi)
        y = y + om * xi
    out = K(y)
    if return_solutions:
        return out, sols
    return out


def deflated_sign_apply(U, v, m0, psi, lam, omega, sigma, tol=1e-13, antiperiodic_t=False):
    """Sec. 1: sign(K) = sum_i psi_i psi_i^dag sign(lambda_i) over the eigenpairs of K, with
    the smallest eigenvectors deflated and the Zolotarev rational applied to the rest:

      sign(K) v ~ sum_i sign(lambda_i) psi_i (psi_i, v) + epsilon(K) (v - sum_i psi_i (psi_i, v))

    psi: (n, ...) orthonormal eigenvectors of K, lam their eigenvalues; omega, sigma the
    rational for the interval left after deflation."""
    v = np.asarray(v)
    proj = v.copy()
    low = np.zeros_like(v)
    for p, l in zip(psi, lam):
        c = vdot(p, v)
        proj = proj - c * p
        low = low + np.sign(l) * c * p
    return low + zolotarev_sign_apply(U, proj, m0, omega, sigma, tol, antiperiodic_t)


def overlap_apply(U, v, m0, mu, omega, sigma, tol=1e-13, antiperiodic_t=False):
    """D(mu) v = 1/2 (1+mu) v + 1/2 (1-mu) gamma5 epsilon(K) v."""
    s = zolotarev_sign_apply(U, v, m0, omega, sigma, tol, antiperiodic_t)
    return 0.5 * (1.0 + mu) * v + 0.5 * (1.0 - mu) * wilson.apply_gamma5(s)


def overlap_apply_dagger(U, v, m0, mu, omega, sigma, tol=1e-13, antiperiodic_t=False):
    """D^dag = gamma5 D gamma5 (gamma5-hermiticity, Sec. 1)."""
    g5 = wilson.apply_gamma5
    return g5(overlap_apply(U, g5(v), m0, mu, omega, sigma, tol, antiperiodic_t))


def free_field_overlap_spectrum(dims, m0, mu, antiperiodic_t=False):
    """Eigenvalues of D(mu) at U = 1 in closed form.

    With gamma5 K = 2 kappa (b + i gamma.s), sign(K) = gamma5 (b + i gamma.s)/sqrt(b^2+s^2),
    so gamma5 sign(K) = (b + i gamma.s)/sqrt(b^2+s^2), whose eigenvalues are
    (b +- i|s|)/sqrt(b^2+|s|^2), each 6-fold per momentum (spin pair x colour).
    """
    lx, ly, lz, lt = dims
    ps = [2 * np.pi * np.arange(L) / L for L in (lx, ly, lz)]
    pt = 2 * np.pi * (np.arange(lt) + (0.5 if antiperiodic_t else 0.0)) / lt
    P = np.meshgrid(ps[0], ps[1], ps[2], pt, indexing="ij")
    b = (sum(1 - np.cos(p) for p in P) - m0).ravel()
    s = np.sqrt(sum(np.sin(p) ** 2 for p in P)).ravel()
    r = np.sqrt(b * b + s * s)
    ev = []
    for sg in (+1, -1):
        lam = 0.5 * (1 + mu) + 0.5 * (1 - mu) * (b + sg * 1j * s) / r
        ev.append(np.repeat(lam, 6))
    return np.concatenate(ev)
