"""CPU-side checks of liboverlap: the library loads, exports every symbol that
include/overlap.h declares, and its host-only numerics agree with the oracle or with
NumPy: the Zolotarev coefficients from its own elliptic-function code, and the small
dense linear algebra the solvers run between launches (Jacobi eigendecomposition,
Cholesky, triangular inverse, pivoted LU, Sturm bisection of a tridiagonal). No GPU
calls."""
import os
import re

import numpy as np
import pytest

from oracle import zolotarev as zo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1501_01855_gb300 import build, binding
    build.build()
    return binding


def test_exports_every_declared_symbol():
    binding = _lib()
    lib = binding.load()
    hdr = open(os.path.join(ROOT, "include", "overlap.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b((?:ovl|overlap|eigsumr)_[a-z0-9_]+)\s*\(", hdr))
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(binding.exported_symbols()) == names


@pytest.mark.parametrize("n,a,b", [(1, 0.2, 2.5), (4, 0.1, 2.5), (16, 0.2136, 2.483), (24, 0.05, 2.54)])
def test_library_zolotarev_matches_oracle(n, a, b):
    binding = _lib()
    om, sg, de = binding.ovl_zolotarev_coeffs(n, a, b)
    o2, s2, d2 = zo.zolotarev(n, a, b)
    assert np.allclose(om, o2, rtol=1e-11, atol=0)
    assert np.allclose(sg, s2, rtol=1e-11, atol=0)
    assert abs(de - d2) <= 1e-6 * d2 + 5e-15


@pytest.mark.parametrize("n,a,b", [(48, 0.002, 2.6), (64, 0.001, 2.6), (64, 0.3, 2.6)])
def test_library_zolotarev_large_order(n, a, b):
    """Up to 64 poles and b/a = 2600 the library's coefficients stay finite and positive
    (plain products of n factors would leave the double range), agree with the oracle's,
    and their sampled error on [a, b] attains the Delta the library reports."""
    binding = _lib()
    om, sg, de = binding.ovl_zolotarev_coeffs(n, a, b)
    assert np.all(np.isfinite(om)) and np.all(om > 0) and np.all(np.diff(sg) > 0)
    o2, s2, _ = zo.zolotarev(n, a, b)
    assert np.allclose(om, o2, rtol=1e-10, atol=0) and np.allclose(sg, s2, rtol=1e-10, atol=0)
    xs = np.exp(np.linspace(np.log(a), np.log(b), 400001))
    err = np.max(np.abs(zo.epsilon(xs, om, sg) - 1.0))
    assert abs(err - de) <= 1e-3 * de + 2e-14, (err, de)


@pytest.mark.parametrize("n,a,b,rtol", [(20, 0.2, 2.6, 1e-14), (64, 0.001, 2.6, 1e-12), (64, 1e-8, 2.6, 1e-7)])
def test_library_zolotarev_sigma_against_mpmath(n, a, b, rtol):
    """sigma_i = a^2 c_{2i-1} from the library's own AGM against 40-digit mpmath, from the
    benchmark's b/a = 13 to b/a = 2.6e8, where 1 - (a/b)^2 rounds to 1 in double; the Delta it
    reports is attained by its own coefficients."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    binding = _lib()
    om, sg, de = binding.ovl_zolotarev_coeffs(n, a, b)
    A, Bv = mp.mpf(a), mp.mpf(b)
    m1 = 1 - (A / Bv) ** 2
    Kp = mp.ellipk(m1)
    for i in range(n):
        u = (2 * i + 1) * Kp / (2 * n)
        ref = float(A * A * mp.ellipfun("sn", u, m=m1) ** 2 / mp.ellipfun("cn", u, m=m1) ** 2)
        assert abs(sg[i] - ref) <= rtol * ref, (i, sg[i], ref)
    assert np.all(np.isfinite(om)) and np.all(om > 0)
    xs = np.exp(np.linspace(np.log(a), np.log(b), 400001))
    err = np.max(np.abs(zo.epsilon(xs, om, sg) - 1.0))
    assert abs(err - de) <= 1e-3 * de + 2e-14, (err, de)


def test_library_rejects_bad_arguments():
    binding = _lib()
    with pytest.raises(binding.OvlError):
        binding.ovl_zolotarev_coeffs(0, 0.1, 1.0)
    with pytest.raises(binding.OvlError):
        binding.ovl_zolotarev_coeffs(4, 1.0, 0.5)


def test_binding_checks_output_buffers():
    """The binding refuses an output that is smaller than the input, of another dtype or
    on the other side of the bus, before any library call (so the library never writes
    past the end of a caller buffer)."""
    binding = _lib()
    x = np.zeros((2, 2, 2, 2, 4, 3), dtype=np.complex128)
    binding._io(None, x, np.zeros_like(x))
    with pytest.raises(ValueError):
        binding._io(None, x, np.zeros((1, 2, 2, 2, 4, 3), dtype=np.complex128))
    with pytest.raises(ValueError):
        binding._io(None, x, np.zeros_like(x, dtype=np.complex64))
    ro = np.zeros_like(x)
    ro.setflags(write=False)
    with pytest.raises(ValueError):
        binding._io(None, x, ro)
    import torch
    with pytest.raises(ValueError):
        binding._io(None, torch.zeros((2, 3), dtype=torch.complex128), torch.zeros((2, 2), dtype=torch.complex128))


# ---- the host numerics the solvers run between launches (Alg. 6, Sec. 4, Sec. 3 bounds)
def _herm(n, rng, spread=1.0):
    Z = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    Q, _ = np.linalg.qr(Z)
    w = np.sort(rng.uniform(-1, 1, n)) * spread
    return (Q * w) @ Q.conj().T, w


@pytest.mark.parametrize("n", [1, 2, 7, 48, 130])
def test_host_eigh_against_numpy(n):
    binding = _lib()
    rng = np.random.default_rng(n)
    A, _ = _herm(n, rng)
    w, Z = binding.ovl_host_eigh(A)
    assert np.all(np.diff(w) >= 0)
    assert np.allclose(w, np.linalg.eigvalsh(A), rtol=0, atol=1e-13 * max(1, n))
    assert np.allclose(Z.conj().T @ Z, np.eye(n), atol=1e-12)
    assert np.allclose(A @ Z, Z * w, atol=1e-12)


def test_host_eigh_degenerate_graded_and_diagonal():
    """Repeated eigenvalues (an invariant subspace, any basis of it), a spectrum spread
    over ten decades as in a Ritz step on D^dag D, and an input that is already diagonal."""
    binding = _lib()
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(9, 9)) + 1j * rng.normal(size=(9, 9)))
    lam = np.array([1, 1, 1, 2, 2, 3, 3, 3, 3], dtype=float)
    A = (Q * lam) @ Q.conj().T
    w, Z = binding.ovl_host_eigh(A)
    assert np.allclose(w, lam, atol=1e-13)
    assert np.allclose(Z.conj().T @ Z, np.eye(9), atol=1e-12)
    assert np.allclose(A @ Z, Z * w, atol=1e-12)
    lam = np.logspace(-8, 2, 24)
    Q, _ = np.linalg.qr(rng.normal(size=(24, 24)) + 1j * rng.normal(size=(24, 24)))
    A = (Q * lam) @ Q.conj().T
    w, Z = binding.ovl_host_eigh(A)
    assert np.allclose(w, lam, rtol=0, atol=1e-12 * lam[-1])
    assert np.allclose(A @ Z, Z * w, atol=1e-12 * lam[-1])
    d = np.array([3.0, -1.0, 2.0, 0.5])
    w, Z = binding.ovl_host_eigh(np.diag(d).astype(complex))
    assert np.array_equal(w, np.sort(d))
    assert np.allclose(np.abs(Z), np.eye(4)[:, np.argsort(d)])


def test_host_eigh_hard_cases():
    """Clusters of equal eigenvalues, a spectrum over 14 decades, an already tridiagonal
    complex matrix, a reducible one, Wilkinson's W (close pairs), rank one and zero; and the
    192 x 192 size of a Ritz step's basis in the deflated 24^3 x 48 solves."""
    binding = _lib()
    rng = np.random.default_rng(8)

    def check(A):
        n = A.shape[0]
        w, Z = binding.ovl_host_eigh(A)
        scale = max(1.0, np.abs(np.linalg.eigvalsh(A)).max())
        assert np.all(np.diff(w) >= 0)
        assert np.allclose(w, np.linalg.eigvalsh(A), rtol=0, atol=1e-13 * scale)
        assert np.abs(Z.conj().T @ Z - np.eye(n)).max() <= 1e-13
        assert np.abs(A @ Z - Z * w).max() <= 1e-13 * scale

    Q, _ = np.linalg.qr(rng.normal(size=(100, 100)) + 1j * rng.normal(size=(100, 100)))
    check((Q * np.repeat([1.0, 2.0, 3.0, 4.0], 25)) @ Q.conj().T)
    check((Q * np.logspace(-12, 2, 100)) @ Q.conj().T)
    T = np.diag(rng.normal(size=50)) + np.diag(rng.normal(size=49) + 1j * rng.normal(size=49), 1)
    T = T + np.triu(T, 1).conj().T
    check(T)
    T[20, 21] = T[21, 20] = 0
    check(T)
    W = np.diag(np.abs(np.arange(-15.0, 16.0))) + np.eye(31, k=1) + np.eye(31, k=-1)
    check(W.astype(complex))
    check(np.ones((40, 40), dtype=complex))
    check(np.zeros((7, 7), dtype=complex))
    Q, _ = np.linalg.qr(rng.normal(size=(192, 192)) + 1j * rng.normal(size=(192, 192)))
    check((Q * np.sort(rng.uniform(1e-4, 3.0, 192))) @ Q.conj().T)


def test_host_cholesky_and_lower_inverse():
    binding = _lib()
    rng = np.random.default_rng(4)
    for n in (1, 5, 64):
        X = rng.normal(size=(n + 3, n)) + 1j * rng.normal(size=(n + 3, n))
        E = X.conj().T @ X                       # a Gram matrix, as in Alg. 6
        L = binding.ovl_host_cholesky(E)
        assert np.allclose(np.triu(L, 1), 0)
        assert np.all(np.real(np.diag(L)) > 0) and np.allclose(np.imag(np.diag(L)), 0)
        assert np.allclose(L @ L.conj().T, E, atol=1e-12 * np.abs(E).max())
        assert np.allclose(L, np.linalg.cholesky(E), atol=1e-11 * np.abs(L).max())
        Li = binding.ovl_host_lower_inverse(L)
        assert np.allclose(Li @ L, np.eye(n), atol=1e-11)
    A, _ = _herm(6, rng)                         # indefinite
    with pytest.raises(binding.OvlError) as e:
        binding.ovl_host_cholesky(A)
    assert e.value.status == binding.OVL_EBREAKDOWN
    with pytest.raises(binding.OvlError) as e:
        binding.ovl_host_lower_inverse(np.zeros((3, 3), dtype=complex))
    assert e.value.status == binding.OVL_EBREAKDOWN


def test_host_lu_solve():
    binding = _lib()
    rng = np.random.default_rng(5)
    for n, nb in ((1, 1), (6, 1), (40, 3)):
        A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        B = rng.normal(size=(n, nb)) + 1j * rng.normal(size=(n, nb))
        X = binding.ovl_host_lu_solve(A, B)
        assert np.allclose(X, np.linalg.solve(A, B), atol=1e-10 * np.abs(X).max())
    # a zero leading entry needs the row exchange
    A = np.array([[0, 1, 2], [3, 0, 1], [1, 1, 0]], dtype=complex)
    b = np.array([1, 2, 3], dtype=complex)
    assert np.allclose(binding.ovl_host_lu_solve(A, b), np.linalg.solve(A, b), atol=1e-14)
    A[:, 1] = 0                                  # a zero pivot column
    with pytest.raises(binding.OvlError) as e:
        binding.ovl_host_lu_solve(A, b)
    assert e.value.status == binding.OVL_EBREAKDOWN


@pytest.mark.parametrize("n", [1, 2, 50, 300])
def test_host_tridiag_extremes(n):
    binding = _lib()
    rng = np.random.default_rng(6 + n)
    d = rng.uniform(0.05, 7.0, n)               # K^2-like: positive diagonal
    e = rng.uniform(0.0, 2.0, n - 1)
    lo, hi = binding.ovl_host_tridiag_extremes(d, e)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    ev = np.linalg.eigvalsh(T)
    assert abs(lo - ev[0]) <= 1e-12 * max(1, abs(ev[-1]))
    assert abs(hi - ev[-1]) <= 1e-12 * max(1, abs(ev[-1]))


def test_host_numerics_reject_bad_arguments():
    binding = _lib()
    lib = binding.load()
    assert lib.ovl_host_eigh(0, None, None, None) == binding.OVL_EINVAL
    assert lib.ovl_host_lu_solve(2, None, None, 1, None) == binding.OVL_EINVAL
    assert lib.ovl_host_tridiag_extremes(3, None, None, None, None) == binding.OVL_EINVAL
    A = np.eye(3, dtype=complex)
    A[1, 2] = np.nan
    with pytest.raises(binding.OvlError) as e:
        binding.ovl_host_eigh(A)
    assert e.value.status == binding.OVL_EINVAL


def test_params_defaults_are_the_documented_ones():
    """ovl_params_default (no GPU) gives the defaults include/overlap.h documents."""
    binding = _lib()
    p = binding.ovl_params_default()
    doc = {"solver": 0, "emulate_fp64": 1, "eta_floor": 1e-2, "sp_switch": 1e-6, "half_switch": 2e-3,
           "relax_factor": 1.0, "gmresr_max": 30, "inner_max": 2000, "mscg_max": 5000, "delta_split": 0.01,
           "c_spec": np.sqrt(3.0) / 2.0, "bc_t": 0, "batch_max": 36, "wilson_variant": -1, "use_graphs": 1,
           "verify": 1, "sign_method": 0, "basis_gb": 96.0, "multimass": 1, "force_pole_group": 0,
           "lanczos_cap": 0, "gram_method": 0}
    for k, v in doc.items():
        assert getattr(p, k) == pytest.approx(v, rel=1e-15), k
    assert not p.stream


def _ritz_setup(k, seed):
    """Gram blocks of a random basis of k vectors on the dense 2^4 overlap operator."""
    from oracle import overlap
    from tests.oracle_util import dense_setup
    mu = 0.05
    _, _, S, _ = dense_setup((2, 2, 2, 2))
    D = overlap.dense_overlap(S, mu, 16)
    G5 = overlap.gamma5_matrix(16)
    rng = np.random.default_rng(seed)
    V = rng.normal(size=(192, k)) + 1j * rng.normal(size=(192, k))
    VD = D @ V
    return mu, D, G5, V, VD, V.conj().T @ V, VD.conj().T @ VD, V.conj().T @ (G5 @ VD)


def test_host_ritz_step_matches_oracle():
    """The library's host algebra of a Ritz step (Alg. 6) on given Gram blocks against the
    oracle's ritz_recalculate on the vectors themselves: Ritz values, residual norms, and the
    Ritz vectors V C (orthonormal, each within a phase of the oracle's)."""
    from oracle import eigen
    binding = _lib()
    delta = 0.01
    for k, keep, seed in ((12, 5, 1), (40, 8, 2)):
        mu, D, G5, V, VD, E, MVD, G5m = _ritz_setup(k, seed)
        ritz, C, res = binding.ovl_host_ritz(E, MVD, G5m, mu, delta, keep)
        lam, Vn, VDn, res_o = eigen.ritz_recalculate(V, VD, mu, delta, keep, (16, 4, 3))
        assert C.shape == (k, keep)
        assert np.allclose(ritz, lam, rtol=1e-11, atol=0)
        assert np.allclose(res, res_o, rtol=1e-8, atol=1e-11)
        W = V @ C
        assert np.allclose(W.conj().T @ W, np.eye(keep), atol=1e-10)
        overlap_ = np.abs(np.sum(W.conj() * Vn, axis=0))
        assert np.allclose(overlap_, 1.0, atol=1e-9)


def test_host_ritz_locally_optimal_restart():
    """restart = 1: the Rayleigh-Ritz of D^dag D + 2 mu delta gamma5 D on the span of the
    lowest keep Ritz vectors of the basis and of the basis without its newest vector
    (2 keep values), against the same construction in NumPy from the oracle's Ritz vectors."""
    from oracle import eigen
    binding = _lib()
    delta, k, keep = 0.01, 30, 6
    mu, D, G5, V, VD, E, MVD, G5m = _ritz_setup(k, 3)
    ritz, C, res = binding.ovl_host_ritz(E, MVD, G5m, mu, delta, keep, restart=True)
    assert len(ritz) == 2 * keep and C.shape == (k, 2 * keep)
    _, V1, _, _ = eigen.ritz_recalculate(V, VD, mu, delta, keep, (16, 4, 3))
    _, V2, _, _ = eigen.ritz_recalculate(V[:, :k - 1], VD[:, :k - 1], mu, delta, keep, (16, 4, 3))
    Qs, _ = np.linalg.qr(np.concatenate([V1, V2], axis=1))
    Mop = D.conj().T @ D + 2 * mu * delta * (G5 @ D)
    ref = np.linalg.eigvalsh(Qs.conj().T @ Mop @ Qs)
    assert np.allclose(ritz, ref, rtol=1e-10, atol=0)
    W = V @ C
    assert np.allclose(W.conj().T @ W, np.eye(2 * keep), atol=1e-9)


def test_host_ritz_without_cholesky_factor():
    """A basis with a repeated vector has a singular E: the step orthonormalises through the
    eigendecomposition of E instead and gives the Ritz values of the span."""
    from oracle import eigen
    binding = _lib()
    delta, keep = 0.01, 5
    mu, D, G5, V, VD, E, MVD, G5m = _ritz_setup(16, 4)
    Vr = np.concatenate([V, V[:, 3:4]], axis=1)
    VDr = D @ Vr
    ritz, C, res = binding.ovl_host_ritz(Vr.conj().T @ Vr, VDr.conj().T @ VDr, Vr.conj().T @ (G5 @ VDr), mu, delta,
                                         keep)
    lam, _, _, _ = eigen.ritz_recalculate(V, VD, mu, delta, keep, (16, 4, 3))
    assert np.allclose(ritz, lam, rtol=1e-8, atol=0)
    W = Vr @ C
    assert np.allclose(W.conj().T @ W, np.eye(keep), atol=1e-8)
    with pytest.raises(binding.OvlError):
        binding.ovl_host_ritz(E, MVD, G5m, mu, delta, 0)


def _sumr_dense(binding, U, rho, b, nsteps):
    """relSUMR on a dense unitary U, A = rho + U: the library's host recurrence for the
    scalars, the vector update of the device kernel written out in NumPy."""
    nb = np.linalg.norm(b)
    q = b / nb
    qt = q.copy()
    p = np.zeros_like(b)
    S = np.zeros_like(b)
    x = np.zeros_like(b)
    state = np.array([0, 0, 0, 0, 1, 0, 1, 0, nb, 0, 0], dtype=np.float64)
    hist = []
    for _ in range(nsteps):
        u = U @ q
        qtu = np.vdot(qt, u)
        dots = [qtu.real, qtu.imag, np.vdot(u, u).real, np.vdot(qt, qt).real]
        R, gs, iR, sp, z, g, gam, isg, sg = binding.ovl_host_sumr_step(rho, dots, state)
        pn = (q - R * p + gs * S) * iR
        S = sp * S + z * p
        p = pn
        x = x + g * pn
        qn = (u + gam * qt) * isg
        qt = sg * qt + np.conj(gam) * qn
        q = qn
        hist.append(abs(complex(state[8], state[9])))
    return x, np.array(hist)


@pytest.mark.parametrize("case", ["random_unitary_200", "overlap_2x2x2x2"])
def test_host_sumr_recurrence_equals_gmres(case):
    """The library's SUMR recurrence (Algs. 1-2 re-derived from App. A) reproduces the
    minimal-residual iterates: on A = rho + U with U a random 200 x 200 unitary and with
    U = gamma5 sign(K) of the 2^4 lattice (rho = (1 + mu)/(1 - mu), mu = 0.05), its residual
    estimate equals the oracle's GMRES residual history and its iterate the GMRES iterate
    (relative 1e-10 over 40 steps); the estimate is the true residual of the iterate."""
    from oracle import solvers
    binding = _lib()
    mu = 0.05
    rho = (1 + mu) / (1 - mu)
    rng = np.random.default_rng(12)
    if case == "random_unitary_200":
        Q, R = np.linalg.qr(rng.normal(size=(200, 200)) + 1j * rng.normal(size=(200, 200)))
        U = Q * (np.diag(R) / np.abs(np.diag(R)))
    else:
        from oracle import overlap
        from tests.oracle_util import dense_setup
        _, _, S, _ = dense_setup((2, 2, 2, 2))
        U = overlap.gamma5_matrix(16) @ S
    N = U.shape[0]
    b = rng.normal(size=N) + 1j * rng.normal(size=N)
    A = rho * np.eye(N) + U
    nsteps = 40
    x, hist = _sumr_dense(binding, U, rho, b, nsteps)
    xg, hg = solvers.minres_iterates(lambda v: A @ v, b, nsteps)
    assert len(hg) == nsteps
    assert np.allclose(hist, hg, rtol=1e-10, atol=1e-13 * np.linalg.norm(b))
    assert np.linalg.norm(x - xg) <= 1e-10 * np.linalg.norm(xg)
    assert abs(np.linalg.norm(b - A @ x) - hist[-1]) <= 1e-10 * np.linalg.norm(b)


def test_host_sumr_step_stops_on_an_exhausted_space():
    """sigma_j = 0 (u in the span of q~_j, an exhausted Krylov space) is OVL_EBREAKDOWN and
    leaves the state as it was."""
    binding = _lib()
    state = np.array([0, 0, 0, 0, 1, 0, 1, 0, 2.0, 0, 0], dtype=np.float64)
    before = state.copy()
    with pytest.raises(binding.OvlError) as e:
        binding.ovl_host_sumr_step(1.1, [1.0, 0.0, 1.0, 1.0], state)   # u = q~: ||u||^2 = |(q~, u)|^2
    assert e.value.status == binding.OVL_EBREAKDOWN
    assert np.array_equal(state, before)


@pytest.mark.parametrize("space", ["exact_low_modes", "random"])
def test_host_deflated_start_matches_oracle(space):
    """The library's deflated start of relSUMR (Sec. 4) from the Gram blocks of a space
    against the oracle's sumr_ls_start on the vectors themselves (2^4, three right-hand sides
    at masses 0.05, 0.3, 0.05): the least-squares x0 and the per-vector form."""
    from oracle import deflation, overlap
    from tests.oracle_util import dense_setup
    binding = _lib()
    _, _, S, _ = dense_setup((2, 2, 2, 2))
    G5 = overlap.gamma5_matrix(16)
    rng = np.random.default_rng(21)
    mus = [0.05, 0.3, 0.05]
    n = 8
    if space == "exact_low_modes":
        H = G5 @ overlap.dense_overlap(S, 0.05, 16)
        w, Yh = np.linalg.eigh(0.5 * (H + H.conj().T))
        Psi = Yh[:, np.argsort(np.abs(w))[:n]]
    else:
        Psi, _ = np.linalg.qr(rng.normal(size=(192, n)) + 1j * rng.normal(size=(192, n)))
    W = G5 @ S @ Psi                                   # w = gamma5 sign(K) psi
    Bs = rng.normal(size=(192, 3)) + 1j * rng.normal(size=(192, 3))
    h = lambda X, Y: X.conj().T @ Y
    blocks = (h(Psi, Psi), h(W, W), h(W, Psi), h(Psi, G5 @ Psi), h(Psi, G5 @ W), h(Psi, Bs), h(W, Bs))
    for per_vector in (False, True):
        co = binding.ovl_host_defl_start(*blocks, mus, per_vector=per_vector)
        for j, mu in enumerate(mus):
            D = overlap.dense_overlap(S, mu, 16)
            shape = (16, 4, 3)
            psi = [Psi[:, i].reshape(shape) for i in range(n)]
            dpsi = [(D @ Psi[:, i]).reshape(shape) for i in range(n)]
            ref = deflation.sumr_ls_start(psi, dpsi, Bs[:, j].reshape(shape), per_vector=per_vector).ravel()
            got = Psi @ co[:, j]
            assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref), (space, per_vector, j)


def test_host_sumr_shared_basis_for_several_masses():
    """Multi-mass relSUMR (Sec. 2: SUMR carries over to many shifts): one Alg. 1 basis
    q_j, q~_j of U serves every mass, each mass with its own recurrence state and its own
    p, S, x; each mass's residual estimate and iterate equal the GMRES iterates of its own
    rho + U (random 200 x 200 unitary, mu = 0.01, 0.02, 0.04)."""
    from oracle import solvers
    binding = _lib()
    rng = np.random.default_rng(13)
    Q, R = np.linalg.qr(rng.normal(size=(200, 200)) + 1j * rng.normal(size=(200, 200)))
    U = Q * (np.diag(R) / np.abs(np.diag(R)))
    b = rng.normal(size=200) + 1j * rng.normal(size=200)
    mus = [0.01, 0.02, 0.04]
    rhos = [(1 + m) / (1 - m) for m in mus]
    nb = np.linalg.norm(b)
    q = b / nb
    qt = q.copy()
    st = [np.array([0, 0, 0, 0, 1, 0, 1, 0, nb, 0, 0], dtype=np.float64) for _ in mus]
    p = [np.zeros_like(b) for _ in mus]
    S = [np.zeros_like(b) for _ in mus]
    x = [np.zeros_like(b) for _ in mus]
    hist = [[] for _ in mus]
    nsteps = 35
    for _ in range(nsteps):
        u = U @ q
        qtu = np.vdot(qt, u)
        dots = [qtu.real, qtu.imag, np.vdot(u, u).real, np.vdot(qt, qt).real]
        for k, rho in enumerate(rhos):
            Rk, gs, iR, sp, z, g, gam, isg, sg = binding.ovl_host_sumr_step(rho, dots, st[k])
            pn = (q - Rk * p[k] + gs * S[k]) * iR
            S[k] = sp * S[k] + z * p[k]
            p[k] = pn
            x[k] = x[k] + g * pn
            hist[k].append(abs(complex(st[k][8], st[k][9])))
        qn = (u + gam * qt) * isg            # the basis step is the same for every mass
        qt = sg * qt + np.conj(gam) * qn
        q = qn
    for k, rho in enumerate(rhos):
        A = rho * np.eye(200) + U
        xg, hg = solvers.minres_iterates(lambda v: A @ v, b, nsteps)
        assert np.allclose(hist[k], hg, rtol=1e-10, atol=1e-13 * nb), k
        assert np.linalg.norm(x[k] - xg) <= 1e-10 * np.linalg.norm(xg), k


def test_host_rayleigh_ritz_of_K():
    """The Rayleigh-Ritz step of the kernel low-mode deflation (Sec. 1) on given Gram blocks
    against SciPy's generalized Hermitian eigensolver: theta in the order of |theta| (signed),
    X C orthonormal, C^dag H C diagonal; exact low eigenvectors of K in the span come out
    exactly among the Ritz pairs; a block with a zero vector (no Cholesky factor of E) is
    OVL_EBREAKDOWN."""
    import scipy.linalg
    from tests.oracle_util import dense_setup
    binding = _lib()
    _, Kd, _, wK = dense_setup((2, 2, 2, 2))
    rng = np.random.default_rng(31)
    m = 14
    X = rng.normal(size=(192, m)) + 1j * rng.normal(size=(192, m))
    E, H = X.conj().T @ X, X.conj().T @ (Kd @ X)
    th, C = binding.ovl_host_rayleigh_ritz(E, H)
    ref = scipy.linalg.eigh(0.5 * (H + H.conj().T), E, eigvals_only=True)
    assert np.allclose(np.sort(th), np.sort(ref), rtol=1e-10, atol=1e-12)
    assert np.all(np.diff(np.abs(th)) >= 0)
    W = X @ C
    assert np.allclose(W.conj().T @ W, np.eye(m), atol=1e-10)
    assert np.allclose(C.conj().T @ H @ C, np.diag(th), atol=1e-10)
    # a block that holds the 4 lowest-|lambda| eigenvectors of K returns them exactly among its
    # Ritz pairs (K is indefinite: the random directions add Ritz values anywhere inside its
    # spectrum, so these need not come first)
    w, Q = np.linalg.eigh(Kd)
    low = Q[:, np.argsort(np.abs(w))[:4]]
    Xl = np.concatenate([low, rng.normal(size=(192, 6)) + 1j * rng.normal(size=(192, 6))], axis=1)
    Xl = Xl @ (rng.normal(size=(10, 10)) + 1j * rng.normal(size=(10, 10)))
    th2, C2 = binding.ovl_host_rayleigh_ritz(Xl.conj().T @ Xl, Xl.conj().T @ (Kd @ Xl))
    Wl = Xl @ C2
    for lam in w[np.argsort(np.abs(w))[:4]]:
        i = int(np.argmin(np.abs(th2 - lam)))
        assert abs(th2[i] - lam) <= 1e-10
        assert np.linalg.norm(Kd @ Wl[:, i] - lam * Wl[:, i]) <= 1e-9
    Xd = X[:, :5].copy()
    Xd[:, 2] = 0.0                          # a zero vector: E has a zero pivot
    with pytest.raises(binding.OvlError) as e:
        binding.ovl_host_rayleigh_ritz(Xd.conj().T @ Xd, Xd.conj().T @ (Kd @ Xd))
    assert e.value.status == binding.OVL_EBREAKDOWN


def test_host_ritz_nearly_dependent_basis():
    """A basis with a vector within 1e-7 or 1e-6 of another (SUMR vectors lose orthogonality
    with an inexact sign, Sec. 5) factorises with a pivot of 1e-14 to 1e-12 of the largest
    diagonal of E. The Ritz step must give the Ritz pairs of the well-conditioned span (the
    orthonormalisation drops the near-null direction); taking U^-1 from such a pivot put
    errors of 6e-3 to 2e-1 into the Ritz values and 1e-2 into the orthonormality."""
    from oracle import eigen
    binding = _lib()
    for seed in range(6):
        for eps in (1e-7, 1e-6):
            mu, D, G5, V, VD, E, MVD, G5m = _ritz_setup(16, 100 + seed)
            rng = np.random.default_rng(seed)
            Vr = np.concatenate([V, V[:, :1] + eps * rng.normal(size=(192, 1))], axis=1)
            VDr = D @ Vr
            ritz, C, res = binding.ovl_host_ritz(Vr.conj().T @ Vr, VDr.conj().T @ VDr, Vr.conj().T @ (G5 @ VDr),
                                                 mu, 0.01, 5)
            lam, _, _, _ = eigen.ritz_recalculate(V, VD, mu, 0.01, 5, (16, 4, 3))
            assert np.allclose(ritz, lam, rtol=1e-7, atol=0), (seed, eps)
            W = Vr @ C
            assert np.allclose(W.conj().T @ W, np.eye(5), atol=1e-9), (seed, eps)


def test_host_ritz_restart_properties_over_random_bases():
    """The locally optimal restart on 20 random bases (k = 14..59, various keep): at least keep
    pairs (near-duplicates of the two Ritz sets are dropped), the lowest keep values at or
    below the Ritz values of the whole basis (the restart span contains those vectors) and
    at or above the true eigenvalues of D^dag D + 2 mu delta gamma5 D, orthonormal vectors,
    and W^dag M W = diag(ritz) exactly (a Rayleigh-Ritz of M on their span)."""
    from oracle import eigen
    binding = _lib()
    for seed in range(20):
        k = int(np.random.default_rng(seed).integers(14, 60))
        keep = int(np.random.default_rng(seed + 99).integers(2, (k - 1) // 2))
        mu, D, G5, V, VD, E, MVD, G5m = _ritz_setup(k, 500 + seed)
        ritz, C, res = binding.ovl_host_ritz(E, MVD, G5m, mu, 0.01, keep, restart=True)
        lam, _, _, _ = eigen.ritz_recalculate(V, VD, mu, 0.01, keep, (16, 4, 3))
        Mop = D.conj().T @ D + 2 * mu * 0.01 * (G5 @ D)
        true = np.linalg.eigvalsh(Mop)
        W = V @ C
        assert keep <= len(ritz) <= 2 * keep, seed
        assert np.all(ritz[:keep] <= lam * (1 + 1e-12) + 1e-14), seed
        assert np.all(ritz >= true[:len(ritz)] - 1e-12), seed
        assert np.abs(W.conj().T @ W - np.eye(len(ritz))).max() <= 1e-10, seed
        assert np.allclose(W.conj().T @ Mop @ W, np.diag(ritz), atol=1e-10), seed


@pytest.mark.parametrize("seed", [12, 13, 14])
def test_host_sumr_estimate_with_an_inexact_sign(seed):
    """With the sign applied inexactly (U + P, ||P|| = eta up to 1e-3: a relaxed sign of Sec. 3),
    the recurrence takes gamma_j as a projection and sigma_j = ||u + gamma_j q~_j||, so that
    V q_j = sigma_j q_{j+1} - gamma_j q~_j holds for the vectors computed (reading 8): its
    residual estimate stays the true residual of the operator it was given, to 1e-2 of itself
    over 60 steps."""
    binding = _lib()
    mu = 0.05
    rho = (1 + mu) / (1 - mu)
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.normal(size=(200, 200)) + 1j * rng.normal(size=(200, 200)))
    U = Q * (np.diag(R) / np.abs(np.diag(R)))
    b = rng.normal(size=200) + 1j * rng.normal(size=200)
    for eta in (1e-6, 1e-4, 1e-3):
        P = rng.normal(size=(200, 200)) + 1j * rng.normal(size=(200, 200))
        P *= eta / np.linalg.norm(P, 2)
        x, hist = _sumr_dense(binding, U + P, rho, b, 60)
        true = np.linalg.norm(b - (rho * np.eye(200) + U + P) @ x)
        assert abs(true - hist[-1]) <= 1e-2 * hist[-1], (eta, true, hist[-1])
