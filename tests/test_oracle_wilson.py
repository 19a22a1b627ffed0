"""Pins of the oracle's Wilson kernel (Sec. 1, aK_xy) against facts fixed by the
paper and by the mathematics: gamma algebra, hermiticity of K = gamma5 D_W,
gauge covariance, the free-field plane-wave spectrum, and a brute-force
site-loop assembly of the defining formula."""
import itertools

import numpy as np
import pytest

import synth
from oracle import wilson


def test_gamma_algebra():
    g, g5 = wilson.GAMMA, wilson.GAMMA5
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4))
        assert np.allclose(g5 @ g[mu] + g[mu] @ g5, 0)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))      # chiral basis


@pytest.mark.parametrize("apt", [False, True])
def test_K_hermitian(apt):
    dims = (4, 4, 4, 4)
    U = synth.gauge_links(dims, 0.3, 7)
    a = synth.gaussian_source(dims, 1)
    b = synth.gaussian_source(dims, 2)
    lhs = np.vdot(a, wilson.apply_K(U, b, 1.4, apt))
    rhs = np.vdot(wilson.apply_K(U, a, 1.4, apt), b)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    U = synth.gauge_links(dims, 0.3, 11)
    rng = np.random.Generator(np.random.PCG64(5))
    Om = synth.random_su3_field(synth.lattice_shape(dims), 2.0, rng)
    Up = np.empty_like(U)
    for mu in range(4):
        Om_f = wilson.shift_links(Om, mu, +1)           # Omega(x+mu)
        Up[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.conj(np.swapaxes(Om_f, -1, -2))
    psi = synth.gaussian_source(dims, 3)
    rot = lambda v: np.einsum("...ab,...sb->...sa", Om, v)
    lhs = wilson.apply_K(Up, rot(psi), 1.4)
    rhs = rot(wilson.apply_K(U, psi, 1.4))
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


@pytest.mark.parametrize("dims,apt", [((2, 2, 2, 2), False), ((2, 2, 2, 4), True), ((4, 2, 2, 2), False)])
def test_free_field_spectrum(dims, apt):
    U = synth.unit_links(dims)
    Kd = wilson.dense_K(U, 1.4, apt)
    ev = np.sort(np.abs(np.linalg.eigvalsh(Kd)))
    ref = wilson.free_field_K_abs_spectrum(dims, 1.4, apt)
    assert np.allclose(ev, ref, atol=1e-13)


def test_free_field_plane_wave():
    """K e^{ipx}u = e^{ipx} 2 kappa gamma5 (b + i gamma.s) u for U = 1."""
    dims = (4, 4, 4, 8)
    m0 = 1.4
    kap = wilson.kappa_of_m(m0)
    n = (1, 3, 2, 5)
    p = [2 * np.pi * n[i] / dims[i] for i in range(4)]
    shp = synth.lattice_shape(dims)
    t, z, y, x = np.meshgrid(*[np.arange(s) for s in shp], indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    rng = np.random.default_rng(0)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi = phase[..., None, None] * u
    out = wilson.apply_K(synth.unit_links(dims), psi, m0)
    b = sum(1 - np.cos(pm) for pm in p) - m0
    M = 2 * kap * wilson.GAMMA5 @ (b * np.eye(4) + 1j * sum(wilson.GAMMA[m] * np.sin(p[m]) for m in range(4)))
    ref = phase[..., None, None] * (M @ u)
    assert np.allclose(out, ref, atol=1e-13)


def test_brute_force_site_loop():
    """Assemble aK_xy with explicit Kronecker deltas over all site pairs (pure Python)."""
    dims = (2, 2, 2, 2)
    lx, ly, lz, lt = dims
    U = synth.gauge_links(dims, 0.5, 21)
    m0 = 1.2
    kap = 1.0 / (8.0 - 2.0 * m0)
    g, g5 = wilson.GAMMA, wilson.GAMMA5
    L = (lx, ly, lz, lt)
    sites = list(itertools.product(range(lt), range(lz), range(ly), range(lx)))
    idx = {s: i for i, s in enumerate(sites)}
    N = len(sites) * 12
    K = np.zeros((N, N), dtype=np.complex128)
    I = np.eye(4)

    def step(s, mu, d):       # s = (t, z, y, x); return s + d*mu
        c = [s[3], s[2], s[1], s[0]]
        c[mu] = (c[mu] + d) % L[mu]
        return (c[3], c[2], c[1], c[0])

    for xs in sites:
        i = idx[xs]
        blk = {xs: np.kron(I, np.eye(3)).astype(np.complex128)}
        for mu in range(4):
            yf = step(xs, mu, +1)
            blk.setdefault(yf, np.zeros((12, 12), complex))
            blk[yf] = blk[yf] - kap * np.kron(I - g[mu], U[xs][mu])
            yb = step(xs, mu, -1)
            blk.setdefault(yb, np.zeros((12, 12), complex))
            blk[yb] = blk[yb] - kap * np.kron(I + g[mu], U[yb][mu].conj().T)
        for ys, B in blk.items():
            j = idx[ys]
            K[i * 12:(i + 1) * 12, j * 12:(j + 1) * 12] += np.kron(g5, np.eye(3)) @ B
    Kd = wilson.dense_K(U, m0)
    assert np.allclose(Kd, K, atol=1e-14)


@pytest.mark.parametrize("apt", [False, True])
def test_site_formula_matches_full_apply(apt):
    dims = (4, 2, 2, 6)
    U = synth.gauge_links(dims, 0.4, 3)
    psi = synth.gaussian_source(dims, 4)
    full = wilson.apply_K(U, psi, 1.3, apt)
    rng = np.random.default_rng(0)
    sites = np.stack([rng.integers(0, d, 20) for d in dims], axis=1)
    sites[0] = (dims[0] - 1, 0, dims[2] - 1, dims[3] - 1)
    sites[1] = (0, 0, 0, 0)
    got = wilson.apply_K_sites(U, psi, 1.3, sites, apt)
    ref = np.array([full[t, z, y, x] for (x, y, z, t) in sites])
    assert np.allclose(got, ref, atol=1e-14)


@pytest.mark.parametrize("dims,apt", [((2, 2, 2, 2), False), ((4, 2, 2, 4), True), ((2, 4, 2, 2), False)])
def test_sparse_K_equals_dense_K(dims, apt):
    """The sparse assembly of K (explicit spin x colour blocks) is the dense operator
    built by applying the formula to unit vectors, including 2-site extents where the
    forward and backward neighbours coincide and the antiperiodic t boundary."""
    U = synth.gauge_links(dims, 0.3, 77)
    Ks = wilson.sparse_K(U, 1.4, apt).toarray()
    Kd = wilson.dense_K(U, 1.4, apt)
    assert np.abs(Ks - Kd).max() <= 1e-14


def test_sparse_K_equals_apply_K_larger():
    dims = (8, 4, 4, 6)
    U = synth.gauge_links(dims, 0.3, 78)
    v = synth.gaussian_source(dims, 79, nvec=2)
    for apt in (False, True):
        K = wilson.sparse_K(U, 1.4, apt)
        for j in range(2):
            got = (K @ v[j].ravel()).reshape(v[j].shape)
            assert np.abs(got - wilson.apply_K(U, v[j], 1.4, apt)).max() <= 1e-13
