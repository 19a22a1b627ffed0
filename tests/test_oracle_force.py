"""Pins of the oracle's gauge-link gradient: central finite differences of S along
random Lie-algebra directions U -> exp(i h X) U, with S evaluated by dense
linear algebra on the frozen Zolotarev rational (2^4 lattice), for the matrix-free
gradient and for its dense form; and the two forms against each other."""
import numpy as np

import synth
from oracle import wilson, overlap, zolotarev as zo, force


def _S_dense(U, phi, m0, mu, om, sg, apt=False):
    Kd = wilson.dense_K(U, m0, apt)
    E = overlap.dense_zolotarev_sign(Kd, om, sg)
    ns = int(np.prod(U.shape[:4]))
    D = overlap.dense_overlap(E, mu, ns)
    x = np.linalg.solve(D.conj().T @ D, phi.ravel())
    return float(np.real(np.vdot(phi.ravel(), x)))


def test_force_finite_differences():
    dims = (2, 2, 2, 2)
    m0, mu = 1.4, 0.05
    U = synth.gauge_links(dims, 0.3, 31)
    phi = synth.gaussian_source(dims, 32)
    om, sg, _ = zo.zolotarev(8, 0.15, 2.6)
    G = force.gradient(U, phi, m0, mu, om, sg, tol=1e-13)
    rng = np.random.Generator(np.random.PCG64(33))
    lam = synth._gell_mann()
    h = 1e-5
    for _ in range(6):
        X = np.einsum("...a,aij->...ij", rng.standard_normal(U.shape[:5] + (8,)), lam) * 0.5
        w, v = np.linalg.eigh(X)
        expo = lambda t: np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * t * w), np.conj(v))
        Sp = _S_dense(expo(h) @ U, phi, m0, mu, om, sg)
        Sm = _S_dense(expo(-h) @ U, phi, m0, mu, om, sg)
        fd = (Sp - Sm) / (2 * h)
        an = 2 * np.real(np.sum(np.conj(G) * (1j * X @ U)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def _fd_check(G, U, phi, m0, mu, om, sg, seed, ndir, apt=False):
    """Central differences of the dense action along ndir random su(3) directions
    against 2 Re <G, i X U>."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = synth._gell_mann()
    h = 1e-5
    for _ in range(ndir):
        X = np.einsum("...a,aij->...ij", rng.standard_normal(U.shape[:5] + (8,)), lam) * 0.5
        w, v = np.linalg.eigh(X)
        expo = lambda t: np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * t * w), np.conj(v))
        Sp = _S_dense(expo(h) @ U, phi, m0, mu, om, sg, apt)
        Sm = _S_dense(expo(-h) @ U, phi, m0, mu, om, sg, apt)
        fd = (Sp - Sm) / (2 * h)
        an = 2 * np.real(np.sum(np.conj(G) * (1j * X @ U)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_dense_gradient_finite_differences():
    """gradient_dense on its own against central differences of the dense action (2^4,
    periodic and antiperiodic in t, two masses)."""
    m0 = 1.4
    om, sg, _ = zo.zolotarev(8, 0.15, 2.6)
    for mu, apt, seed in ((0.05, False, 41), (0.3, True, 42)):
        U = synth.gauge_links((2, 2, 2, 2), 0.3, seed)
        phi = synth.gaussian_source((2, 2, 2, 2), seed + 1)
        G, _ = force.gradient_dense(U, phi, m0, mu, om, sg, antiperiodic_t=apt)
        _fd_check(G, U, phi, m0, mu, om, sg, seed + 2, 4, apt)


def test_dense_gradient_equals_matrix_free():
    """gradient_dense (dense K, eigendecomposition) and gradient (matrix-free CGs) are the
    same formula: on 2^4, periodic and antiperiodic in t, they agree, and its
    action equals the dense D^dag D solve."""
    m0, mu = 1.4, 0.05
    om, sg, _ = zo.zolotarev(8, 0.15, 2.6)
    for dims, apt in (((2, 2, 2, 2), False), ((2, 2, 2, 2), True)):
        U = synth.gauge_links(dims, 0.3, 61)
        phi = synth.gaussian_source(dims, 62)
        G1 = force.gradient(U, phi, m0, mu, om, sg, tol=1e-14, antiperiodic_t=apt)
        G2, S2 = force.gradient_dense(U, phi, m0, mu, om, sg, antiperiodic_t=apt)
        assert np.linalg.norm(G1 - G2) <= 1e-9 * np.linalg.norm(G2)
        S1, _ = force.action(U, phi, m0, mu, om, sg, tol=1e-14, antiperiodic_t=apt)
        assert abs(S1 - S2) <= 1e-10 * abs(S2)
    U = synth.gauge_links((2, 2, 2, 2), 0.3, 61)
    phi = synth.gaussian_source((2, 2, 2, 2), 62)
    assert abs(force.gradient_dense(U, phi, m0, mu, om, sg)[1] - _S_dense(U, phi, m0, mu, om, sg)) <= 1e-10 * abs(
        _S_dense(U, phi, m0, mu, om, sg))


def test_matrix_free_gradient_quick():
    """The matrix-free gradient (CG solves at 1e-9) equals the dense form to 1e-6 on 2^4
    with a 4-pole rational, and the action to 1e-7: the quick form of the check above, cheap
    enough to rerun under planted mistakes."""
    m0, mu = 1.4, 0.05
    om, sg, _ = zo.zolotarev(4, 0.15, 2.6)
    U = synth.gauge_links((2, 2, 2, 2), 0.3, 61)
    phi = synth.gaussian_source((2, 2, 2, 2), 62)
    G1 = force.gradient(U, phi, m0, mu, om, sg, tol=1e-9)
    G2, S2 = force.gradient_dense(U, phi, m0, mu, om, sg)
    assert np.linalg.norm(G1 - G2) <= 1e-6 * np.linalg.norm(G2)
    S1, _ = force.action(U, phi, m0, mu, om, sg, tol=1e-9)
    assert abs(S1 - S2) <= 1e-7 * abs(S2)
