"""Planted mistakes in the oracle: every pin must be able to fail.

Each case rewrites one expression of one oracle function into a plausible wrong form
(a flipped sign, a dropped term or factor, a missing conjugation, a transposed or
shifted operand, a wrong index), loads the rewritten function into its module for
the duration of the case, and runs the listed pins of tests/test_oracle_*.py. The
case passes when at least one of them fails. The expression to rewrite must occur
exactly once in the function's source, so a later change of the oracle that moves it
shows up here as an error, not as a silent pass.

The planted code lives only in this process, on the CPU; the oracle's files are not
touched. A rewrite that leaves every output unchanged in exact arithmetic is no case:
dropping the conjugate in the q-tilde update of eigsumr_build changes the basis vectors
but not their span (each new one still adds U q_j), so the Rayleigh-Ritz result of
Alg. 6 is the same; the same rewrite in sumr_basis, whose basis is an output, is a
case. Neither is a rewrite that keeps an iteration from converging (gamma5 dropped from
H, whose square then is no CG operator): it is caught only after its solves reach their
iteration limits, minutes later. Pins that run the oracle in a spawn process pool (the workers import the
unmodified oracle) and the minute-long matrix-free force pins are not used here: the
matrix-free gradient is checked by the quick form of its equality with the dense
gradient, whose own mistakes are caught by finite differences.
"""
import inspect
import textwrap

import numpy as np
import pytest

from oracle import deflation, eigen, force, overlap, solvers, wilson, zolotarev
from tests import oracle_util
from tests import test_oracle_eigen_deflation as te
from tests import test_oracle_force as tf
from tests import test_oracle_overlap as to
from tests import test_oracle_solvers as ts
from tests import test_oracle_wilson as tw
from tests import test_oracle_zolotarev as tz

PINS = {
    # Wilson kernel, Sec. 1 (aK_xy)
    "K hermitian": lambda: tw.test_K_hermitian(False),
    "K hermitian, antiperiodic t": lambda: tw.test_K_hermitian(True),
    "gauge covariance": tw.test_gauge_covariance,
    "free-field plane wave": tw.test_free_field_plane_wave,
    "free-field |lambda(K)| 2^4": lambda: tw.test_free_field_spectrum((2, 2, 2, 2), False),
    "brute-force site loop": tw.test_brute_force_site_loop,
    "site formula": lambda: tw.test_site_formula_matches_full_apply(False),
    "site formula, antiperiodic t": lambda: tw.test_site_formula_matches_full_apply(True),
    "sparse K = dense K, 2^4": lambda: tw.test_sparse_K_equals_dense_K((2, 2, 2, 2), False),
    "sparse K = dense K, 4x2x2x4 antiperiodic": lambda: tw.test_sparse_K_equals_dense_K((4, 2, 2, 4), True),
    "sparse K = dense K, 2x4x2x2": lambda: tw.test_sparse_K_equals_dense_K((2, 4, 2, 2), False),
    "sparse K = apply_K, 8x4x4x6": tw.test_sparse_K_equals_apply_K_larger,
    # Zolotarev rational, Sec. 3
    "n = 1 closed form": lambda: tz.test_n1_closed_form(0.2, 2.5),
    "equioscillation n = 2": lambda: tz.test_equioscillation(2, 0.2, 2.5),
    "equioscillation n = 3": lambda: tz.test_equioscillation(3, 0.2, 2.5),
    "Delta monotone, epsilon odd": tz.test_delta_monotone_and_odd,
    # sign function and overlap operator, Secs. 1, 3
    "sign^2 = 1": to.test_sign_squares_to_one,
    "Zolotarev bound, per-pole CG": to.test_zolotarev_bound_and_per_pole_cg,
    "Ginsparg-Wilson": to.test_ginsparg_wilson,
    "gamma5-hermiticity, circle, mu = 0.3": lambda: to.test_gamma5_hermiticity_circle_normality(0.3),
    "free-field overlap spectrum 2^4": lambda: to.test_free_field_overlap_spectrum((2, 2, 2, 2), False),
    "matrix-free D = dense D": to.test_matrix_free_overlap_matches_dense,
    "deflated sign": to.test_deflated_sign_pins,
    "batched forms = dense rational": to.test_batched_forms_in_process_match_dense,
    # solvers, Algs. 1-4
    "Alg. 1 basis": ts.test_alg1_basis,
    "minimal residual = brute force": ts.test_minres_iterates_brute_force,
    "GMRESR, inexact inner": ts.test_gmresr_inexact_inner_monotone,
    "CGNE, spectral preconditioner": ts.test_cgne_spectral_with_exact_eigenvectors,
    "restarted GMRES = dense solve": ts.test_gmres_solve_matches_dense_solve,
    # eigen accumulation and deflation, Secs. 4-5
    "Ritz step, exact in subspace": te.test_ritz_exact_in_subspace_and_interlacing,
    "eigSUMR = Rayleigh-Ritz": te.test_eigsumr_equals_rayleigh_ritz_on_krylov_space,
    "Galerkin and LS starts": te.test_galerkin_and_ls_starts,
    "spectral preconditioner c^2": te.test_spectral_preconditioner_maps_to_c2,
    # force
    "dense gradient, finite differences": tf.test_dense_gradient_finite_differences,
    "matrix-free gradient = dense gradient": tf.test_matrix_free_gradient_quick,
}

# (module, function, expression, planted form, pins that may catch it)
CASES = [
    # ---- wilson.hopping: the four hop terms of aK_xy
    (wilson, "hopping", "I4 - GAMMA[mu], fwd", "I4 + GAMMA[mu], fwd",
     ["brute-force site loop", "free-field plane wave"]),
    (wilson, "hopping", "I4 + GAMMA[mu], bwd", "I4 - GAMMA[mu], bwd",
     ["K hermitian", "brute-force site loop"]),
    (wilson, "hopping", '"...ba,...sb->...sa", np.conj(Ub)', '"...ab,...sb->...sa", np.conj(Ub)',
     ["K hermitian", "brute-force site loop"]),
    (wilson, "hopping", "np.conj(Ub), shift", "Ub, shift", ["K hermitian", "brute-force site loop"]),
    (wilson, "hopping", "Ub = shift_links(Umu, mu, -1)", "Ub = Umu", ["gauge covariance", "K hermitian"]),
    (wilson, "hopping", "Umu, shift(psi, mu, +1, antiperiodic_t)",
     "shift_links(Umu, mu, +1), shift(psi, mu, +1, antiperiodic_t)", ["gauge covariance", "K hermitian"]),
    (wilson, "hopping", "shift(psi, mu, -1, antiperiodic_t)", "shift(psi, mu, +1, antiperiodic_t)",
     ["K hermitian", "brute-force site loop"]),
    # ---- wilson: kappa, gamma5, shifts and the antiperiodic boundary
    (wilson, "kappa_of_m", "8.0 - 2.0 * m0", "8.0 + 2.0 * m0",
     ["free-field plane wave", "free-field |lambda(K)| 2^4"]),
    (wilson, "kappa_of_m", "1.0 / (8.0 - 2.0 * m0)", "1.0 / (4.0 - m0)",
     ["free-field plane wave", "brute-force site loop"]),
    (wilson, "apply_K", "apply_gamma5(psi - kap * hopping(U, psi, antiperiodic_t))",
     "psi - kap * hopping(U, psi, antiperiodic_t)", ["K hermitian", "brute-force site loop"]),
    (wilson, "apply_K", "psi - kap * hopping", "psi + kap * hopping",
     ["brute-force site loop", "free-field plane wave"]),
    (wilson, "shift", "np.roll(psi, -sign, axis=ax)", "np.roll(psi, sign, axis=ax)",
     ["brute-force site loop", "free-field plane wave"]),
    (wilson, "shift", "idx[ax] = n - 1 if sign > 0 else 0", "idx[ax] = 0 if sign > 0 else n - 1",
     ["K hermitian, antiperiodic t", "site formula, antiperiodic t"]),
    (wilson, "shift_links", "np.roll(U_mu, -sign, axis=ax)", "np.roll(U_mu, sign, axis=ax)",
     ["K hermitian", "brute-force site loop"]),
    # ---- wilson: the independent assemblies (site formula, sparse K) and the closed form
    (wilson, "apply_K_sites", "(pf @ Uf.T)", "(pf @ Uf)", ["site formula"]),
    (wilson, "apply_K_sites", "(pb @ np.conj(Ub))", "(pb @ Ub)", ["site formula"]),
    (wilson, "apply_K_sites", "c[3] == L[3] - 1", "c[3] == 0", ["site formula, antiperiodic t"]),
    (wilson, "sparse_K", '"st,xba->xsatb", Pp', '"st,xab->xsatb", Pp', ["sparse K = dense K, 2^4"]),
    (wilson, "sparse_K", "bwd = np.roll(site, +1, axis=ax).ravel()", "bwd = np.roll(site, -1, axis=ax).ravel()",
     ["sparse K = dense K, 2x4x2x2", "sparse K = apply_K, 8x4x4x6"]),
    (wilson, "sparse_K", "sb[tco == 0] = -1.0", "sb[tco == lt - 1] = -1.0",
     ["sparse K = dense K, 4x2x2x4 antiperiodic", "sparse K = apply_K, 8x4x4x6"]),
    (wilson, "sparse_K", "np.kron(GAMMA5, np.eye(3))", "np.kron(I4, np.eye(3))", ["sparse K = dense K, 2^4"]),
    (wilson, "dense_operator", "return cols.reshape(n, n).T.copy()", "return cols.reshape(n, n).copy()",
     ["sparse K = dense K, 2^4", "free-field |lambda(K)| 2^4"]),
    (wilson, "free_field_K_abs_spectrum", "lam = 2 * kap * np.sqrt(b ** 2 + s2)", "lam = kap * np.sqrt(b ** 2 + s2)",
     ["free-field |lambda(K)| 2^4"]),
    # ---- zolotarev: elliptic coefficients, product form, partial fractions
    (zolotarev, "c_coefficients", "m1 = 1.0 - k * k", "m1 = k * k",
     ["n = 1 closed form", "equioscillation n = 3"]),
    (zolotarev, "c_coefficients", "l[near] * Kp / (2 * n)", "l[near] * Kp / n",
     ["n = 1 closed form", "equioscillation n = 3"]),
    (zolotarev, "c_coefficients", "special.ellipkm1(k * k)", "special.ellipkm1(1.0 - k * k)",
     ["n = 1 closed form", "equioscillation n = 3"]),
    (zolotarev, "c_coefficients", "(cn / (k * sn)) ** 2", "(cn / sn) ** 2", ["equioscillation n = 3"]),
    (zolotarev, "c_coefficients", "(2 * n - l[~near])", "(2 * n - l[~near] + 1)", ["equioscillation n = 3"]),
    (zolotarev, "c_coefficients", "sn ** 2 / cn ** 2", "cn ** 2 / sn ** 2",
     ["n = 1 closed form", "equioscillation n = 3"]),
    (zolotarev, "r0", "r = r * (y2 + c[2 * l - 1]) / (y2 + c[2 * l - 2])",
     "r = r * (y2 + c[2 * l - 2]) / (y2 + c[2 * l - 2])", ["equioscillation n = 3"]),
    (zolotarev, "r0", "r = y / (y2 + c[2 * n - 2])", "r = y / (y2 + c[2 * n - 3])", ["equioscillation n = 3"]),
    (zolotarev, "zolotarev", "d = 2.0 / (lo + hi)", "d = 1.0 / hi", ["n = 1 closed form", "equioscillation n = 3"]),
    (zolotarev, "zolotarev", "omega[i] = a * d * ratio", "omega[i] = d * ratio",
     ["n = 1 closed form", "equioscillation n = 3"]),
    (zolotarev, "zolotarev", "sigma = a * a * codd", "sigma = a * codd",
     ["n = 1 closed form", "equioscillation n = 3"]),
    (zolotarev, "zolotarev", "others - codd[i]", "codd[i] - others",
     ["equioscillation n = 2", "Delta monotone, epsilon odd"]),
    (zolotarev, "zolotarev", "zip(ceven - codd[i]", "zip(codd[i] - ceven",
     ["equioscillation n = 2", "Delta monotone, epsilon odd"]),
    (zolotarev, "zolotarev", "delta = (hi - lo) / (hi + lo)", "delta = (hi - lo) / hi",
     ["n = 1 closed form", "equioscillation n = 3"]),
    (zolotarev, "epsilon", "w * x / (x * x + s)", "w / (x * x + s)", ["equioscillation n = 3"]),
    # ---- overlap: spectral sign, D(mu), matrix-free rational
    (overlap, "dense_sign", "(Q * np.sign(w)) @ np.conj(Q.T)", "(Q * np.sign(w)) @ Q.T", ["sign^2 = 1"]),
    (overlap, "dense_zolotarev_sign", "om * w / (w * w + s)", "om / (w * w + s)",
     ["Zolotarev bound, per-pole CG"]),
    (overlap, "dense_overlap", "0.5 * (1.0 + mu) * np.eye(n) + 0.5 * (1.0 - mu) * (G5 @ Sd)",
     "0.5 * (1.0 - mu) * np.eye(n) + 0.5 * (1.0 + mu) * (G5 @ Sd)",
     ["gamma5-hermiticity, circle, mu = 0.3", "free-field overlap spectrum 2^4"]),
    (overlap, "dense_overlap", "0.5 * (1.0 - mu) * (G5 @ Sd)", "(1.0 - mu) * (G5 @ Sd)",
     ["Ginsparg-Wilson", "gamma5-hermiticity, circle, mu = 0.3"]),
    (overlap, "dense_overlap", "(G5 @ Sd)", "(Sd @ G5)", ["matrix-free D = dense D"]),
    (overlap, "gamma5_matrix", "np.kron(g5, np.eye(3))", "np.kron(np.eye(3), g5)",
     ["matrix-free D = dense D", "Ginsparg-Wilson"]),
    (overlap, "cg", "x = x + alpha * p", "x = x + alpha * r", ["Zolotarev bound, per-pole CG"]),
    (overlap, "zolotarev_sign_apply", "out = K(y)", "out = y", ["Zolotarev bound, per-pole CG"]),
    (overlap, "zolotarev_sign_apply", "y = y + om * xi", "y = y + xi", ["Zolotarev bound, per-pole CG"]),
    (overlap, "overlap_apply", "0.5 * (1.0 + mu) * v + 0.5 * (1.0 - mu) * wilson.apply_gamma5(s)",
     "0.5 * (1.0 - mu) * v + 0.5 * (1.0 + mu) * wilson.apply_gamma5(s)", ["matrix-free D = dense D"]),
    (overlap, "overlap_apply", "wilson.apply_gamma5(s)", "s", ["matrix-free D = dense D"]),
    (overlap, "overlap_apply_dagger", "g5(overlap_apply(U, g5(v),", "(overlap_apply(U, (v),",
     ["matrix-free D = dense D"]),
    (overlap, "_worker_pole_solve", "K @ (K @ p) + s * p", "K @ p + s * p", ["batched forms = dense rational"]),
    (overlap, "shifted_solves", "xs = [[res[j * npol + i][0]", "xs = [[res[i * nv + j][0]",
     ["batched forms = dense rational"]),
    (overlap, "zolotarev_sign_apply_many", "out[j] = (K @ y).reshape(vs.shape[1:])", "out[j] = y.reshape(vs.shape[1:])",
     ["batched forms = dense rational"]),
    (overlap, "zolotarev_sign_apply_many", "y = sum(om * x for om, x in zip(omega, xs[j]))",
     "y = sum(om * x for om, x in zip(omega, xs[0]))", ["batched forms = dense rational"]),
    (overlap, "overlap_apply_many", "0.5 * (1.0 + mus[j]) * vs[j] + 0.5 * (1.0 - mus[j])",
     "0.5 * (1.0 + mus[0]) * vs[j] + 0.5 * (1.0 - mus[0])", ["batched forms = dense rational"]),
    (overlap, "deflated_sign_apply", "c = vdot(p, v)", "c = vdot(v, p)", ["deflated sign"]),
    (overlap, "deflated_sign_apply", "proj = proj - c * p", "proj = proj", ["deflated sign"]),
    (overlap, "deflated_sign_apply", "low = low + np.sign(l) * c * p", "low = low + c * p", ["deflated sign"]),
    (overlap, "free_field_overlap_spectrum", "(b + sg * 1j * s) / r", "(b + sg * 1j * s)",
     ["free-field overlap spectrum 2^4"]),
    # ---- solvers: Alg. 1 recurrence, minimal residual, GMRESR, CGNE
    (solvers, "vdot", "np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel())",
     "np.dot(np.asarray(a).ravel(), np.asarray(b).ravel())", ["Alg. 1 basis", "minimal residual = brute force"]),
    (solvers, "sumr_basis", "qt = s * qt + np.conj(g) * qn", "qt = s * qt + g * qn", ["Alg. 1 basis"]),
    (solvers, "sumr_basis", "g = -vdot(qt, u)", "g = vdot(qt, u)", ["Alg. 1 basis"]),
    (solvers, "sumr_basis", "qn = (u + g * qt) / s", "qn = (u - g * qt) / s", ["Alg. 1 basis"]),
    (solvers, "minres_iterates", "h = vdot(V[i], w)", "h = vdot(w, V[i])", ["minimal residual = brute force"]),
    (solvers, "minres_iterates", "e1[0] = beta", "e1[0] = 1.0", ["minimal residual = brute force"]),
    (solvers, "gmres_solve", "if norm(r) <= tol * nb:", "if norm(r) <= tol * nb or it > 0:",
     ["restarted GMRES = dense solve"]),
    (solvers, "gmresr", "alpha = vdot(c, r)", "alpha = vdot(r, c)", ["GMRESR, inexact inner"]),
    (solvers, "gmresr", "u = u - beta * uj", "u = u", ["GMRESR, inexact inner"]),
    (solvers, "gmresr", "u = u / nu", "u = u", ["GMRESR, inexact inner"]),
    (solvers, "cgne_spectral", "return applyH(apply_Hhat_inv(x)), j", "return applyH(x), j",
     ["CGNE, spectral preconditioner"]),
    (solvers, "cgne_spectral", "r = apply_Hhat_inv(b)", "r = b.copy()", ["CGNE, spectral preconditioner"]),
    # ---- eigen: Alg. 6 (Ritz step) and Alg. 5 (eigSUMR build)
    (eigen, "ritz_recalculate", " + 2.0 * mu * delta * (np.conj(Vm.T) @ g5VD)", "",
     ["Ritz step, exact in subspace", "eigSUMR = Rayleigh-Ritz"]),
    (eigen, "ritz_recalculate", "T = Linv @ M @ Uinv", "T = Uinv @ M @ Linv",
     ["Ritz step, exact in subspace", "eigSUMR = Rayleigh-Ritz"]),
    (eigen, "ritz_recalculate", "C = Uinv @ Y[:, :n_keep]", "C = Y[:, :n_keep]",
     ["Ritz step, exact in subspace", "eigSUMR = Rayleigh-Ritz"]),
    (eigen, "ritz_recalculate", "r = g5vd - Vn[:, i] * np.vdot(Vn[:, i], g5vd)", "r = g5vd - Vn[:, i]",
     ["eigSUMR = Rayleigh-Ritz"]),
    (eigen, "eigsumr_build", "0.5 * (1 - mu) * u + 0.5 * (1 + mu) * q", "0.5 * (1 + mu) * u + 0.5 * (1 - mu) * q",
     ["eigSUMR = Rayleigh-Ritz"]),
    (eigen, "eigsumr_build", "V.append(q.ravel())", "V.append(u.ravel())", ["eigSUMR = Rayleigh-Ritz"]),
    # ---- deflation: Galerkin / least-squares starts, spectral preconditioner (Sec. 4)
    (deflation, "galerkin_start", "np.linalg.solve(G, np.conj(Vm.T) @ r)", "np.linalg.solve(G, Vm.T @ r)",
     ["Galerkin and LS starts"]),
    (deflation, "galerkin_start", "G = np.conj(Vm.T) @ AV", "G = np.conj(Vm.T) @ Vm", ["Galerkin and LS starts"]),
    (deflation, "sumr_ls_start", "np.linalg.solve(G, np.conj(DP.T) @ bb)", "np.linalg.solve(G, DP.T @ bb)",
     ["Galerkin and LS starts"]),
    (deflation, "sumr_ls_start", "DP = DVm @ Y", "DP = DVm", ["Galerkin and LS starts"]),
    (deflation, "sumr_ls_start", "np.vdot(DP[:, j], bb) / np.vdot", "np.vdot(bb, DP[:, j]) / np.vdot",
     ["Galerkin and LS starts"]),
    (deflation, "spectral_precond", "c / np.sqrt(np.asarray(mus, dtype=np.float64)) - 1.0",
     "c / np.asarray(mus, dtype=np.float64) - 1.0",
     ["spectral preconditioner c^2", "CGNE, spectral preconditioner"]),
    (deflation, "spectral_precond", "(np.conj(Vm.T) @ xs)", "(Vm.T @ xs)",
     ["spectral preconditioner c^2", "CGNE, spectral preconditioner"]),
    # ---- force: the link outer products and the dense gradient
    (force, "link_outer", "np.conj(F) + np.swapaxes(G, -1, -2)", "F + np.swapaxes(G, -1, -2)",
     ["dense gradient, finite differences"]),
    (force, "link_outer", "P1 = g5 @ (wilson.I4 - wilson.GAMMA[mu])", "P1 = g5 @ (wilson.I4 + wilson.GAMMA[mu])",
     ["dense gradient, finite differences"]),
    (force, "link_outer", "-0.5 * kap", "-kap", ["dense gradient, finite differences"]),
    (force, "link_outer", "xf = wilson.shift(x, mu, +1, antiperiodic_t)", "xf = x",
     ["dense gradient, finite differences"]),
    (force, "gradient_dense", "- link_outer(r(Kd @ b), r(a), m0, antiperiodic_t))",
     "+ link_outer(r(Kd @ b), r(a), m0, antiperiodic_t))", ["dense gradient, finite differences"]),
    (force, "gradient_dense", "c = -(1.0 - mu) * om", "c = -(1.0 + mu) * om", ["dense gradient, finite differences"]),
    (force, "gradient_dense", "Ri @ Kpsi", "Ri @ psi", ["dense gradient, finite differences"]),
    (force, "gradient", "- link_outer(b, Ka, m0, antiperiodic_t)", "+ link_outer(b, Ka, m0, antiperiodic_t)",
     ["matrix-free gradient = dense gradient"]),
    (force, "gradient", "b, _ = overlap.cg(A, Kpsi, tol)", "b, _ = overlap.cg(A, psi, tol)",
     ["matrix-free gradient = dense gradient"]),
    (force, "gradient", "psi = apply_H(U, chi, m0, mu, omega, sigma, tol, antiperiodic_t)", "psi = chi",
     ["matrix-free gradient = dense gradient"]),
    (force, "action", "overlap.vdot(phi, chi)", "overlap.vdot(chi, chi)", ["matrix-free gradient = dense gradient"]),
]


@pytest.fixture
def fresh_cache():
    """The dense 2^4 set-up is cached; a planted mistake must neither see the correct
    cached operators nor leave its own behind."""
    oracle_util.dense_setup.cache_clear()
    yield
    oracle_util.dense_setup.cache_clear()


def _plant(monkeypatch, module, name, expr, planted):
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    n = src.count(expr)
    assert n == 1, "%s.%s: expression %r occurs %d times" % (module.__name__, name, expr, n)
    code = compile(src.replace(expr, planted), "<planted %s.%s>" % (module.__name__, name), "exec")
    scope = {}
    exec(code, module.__dict__, scope)
    monkeypatch.setattr(module, name, scope[name])


def _first_failing(pins):
    """Name of the first pin that fails, else None. A pin fails by an assertion, or by a
    linear-algebra error (a Cholesky or solve of a matrix the mistake made singular or
    indefinite)."""
    for name in pins:
        try:
            with np.errstate(all="ignore"):
                PINS[name]()
        except (AssertionError, np.linalg.LinAlgError):
            return name
    return None


def _case_id(c):
    module, name, expr, planted, _ = c
    return "%s.%s:%s->%s" % (module.__name__.split(".")[-1], name, expr.strip()[:32], planted.strip()[:32])


def test_pins_pass_unplanted(fresh_cache):
    """The pins used below pass on the oracle as written (so a failure under a planted
    mistake is the mistake's doing)."""
    used = sorted({p for c in CASES for p in c[4]})
    assert set(used) <= set(PINS)
    assert _first_failing(used) is None


@pytest.mark.parametrize("case", CASES, ids=[_case_id(c) for c in CASES])
def test_planted_mistake_is_caught(case, monkeypatch, fresh_cache):
    module, name, expr, planted, pins = case
    _plant(monkeypatch, module, name, expr, planted)
    assert _first_failing(pins) is not None, "no pin caught %s.%s: %r -> %r" % (module.__name__, name, expr, planted)


def test_planted_axis_map_is_caught(monkeypatch, fresh_cache):
    """Directions mapped to the wrong lattice axes (x and y exchanged) in the Wilson kernel."""
    monkeypatch.setattr(wilson, "MU_AXIS", {0: 2, 1: 3, 2: 1, 3: 0})
    assert _first_failing(["brute-force site loop", "free-field plane wave"]) is not None
