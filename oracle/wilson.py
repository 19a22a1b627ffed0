"""Wilson kernel of the overlap operator, written out from Sec. 1 (the equation
for aK_xy):

  K psi(x) = gamma5 [ psi(x) - kappa sum_mu ( (1-gamma_mu) U_mu(x) psi(x+mu)
                                             + (1+gamma_mu) U_mu(x-mu)^dag psi(x-mu) ) ]

with kappa = 1/(8-2m). The gamma matrices are the Hermitian chiral
(DeGrand-Rossi) set; the paper fixes only "the standard Hermitian form" with
gamma_mu^2 = 1, and every pin used here is basis independent.

No spin projection, no link compression, no blocking: explicit 4x4 spin
matrices and 3x3 colour matrices applied with einsum. Test infrastructure only.
"""
import numpy as np

# site axes of the canonical array (Lt, Lz, Ly, Lx): direction mu -> numpy axis
MU_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}

I4 = np.eye(4, dtype=np.complex128)


def gamma_matrices():
    """(gamma_1..gamma_4, gamma_5) in the DeGrand-Rossi chiral basis."""
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    i = 1j
    g[0] = [[0, 0, 0, i], [0, 0, i, 0], [0, -i, 0, 0], [-i, 0, 0, 0]]
    g[1] = [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]]
    g[2] = [[0, 0, i, 0], [0, 0, 0, -i], [-i, 0, 0, 0], [0, i, 0, 0]]
    g[3] = [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]]
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


GAMMA, GAMMA5 = gamma_matrices()


def kappa_of_m(m0):
    """kappa = 1/(8 - 2m), Sec. 1."""
    return 1.0 / (8.0 - 2.0 * m0)


def shift(psi, mu, sign, antiperiodic_t=False):
    """Return psi(x + sign*mu) for psi with site axes (..., Lt, Lz, Ly, Lx, ...).

    psi has shape (..., Lt, Lz, Ly, Lx, 4, 3) or links (..., Lt, Lz, Ly, Lx, 3, 3):
    the site axes are found counting from the end (two internal axes).
    """
    ax = psi.ndim - 6 + MU_AXIS[mu]
    out = np.roll(psi, -sign, axis=ax)
    if antiperiodic_t and mu == 3:
        n = psi.shape[ax]
        idx = [slice(None)] * psi.ndim
        # the wrapped slice: for +t it is the last time slice, for -t the first
        idx[ax] = n - 1 if sign > 0 else 0
        out[tuple(idx)] *= -1.0
    return out


def shift_links(U_mu, mu, sign):
    """U_mu(x + sign*mu-hat) for one link direction with axes (Lt, Lz, Ly, Lx, 3, 3)."""
    ax = MU_AXIS[mu]
    return np.roll(U_mu, -sign, axis=ax)


def hopping(U, psi, antiperiodic_t=False):
    """sum_mu (1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)."""
    out = np.zeros_like(psi)
    for mu in range(4):
        Umu = U[..., mu, :, :]
        fwd = np.einsum("...ab,...sb->...sa", Umu, shift(psi, mu, +1, antiperiodic_t))
        out += np.einsum("st,...tb->...sb", I4 - GAMMA[mu], fwd)
        Ub = shift_links(Umu, mu, -1)                       # U_mu(x - mu)
        bwd = np.einsum("...ba,...sb->...sa", np.conj(Ub), shift(psi, mu, -1, antiperiodic_t))
        out += np.einsum("st,...tb->...sb", I4 + GAMMA[mu], bwd)
    return out


def apply_gamma5(psi):
    return np.einsum("st,...tb->...sb", GAMMA5, psi)


def apply_K(U, psi, m0, antiperiodic_t=False):
    """K psi = gamma5 [psi - kappa * hopping(psi)]   (Sec. 1, aK_xy)."""
    kap = kappa_of_m(m0)
    return apply_gamma5(psi - kap * hopping(U, psi, antiperiodic_t))


def apply_DW(U, psi, m0, antiperiodic_t=False):
    """gamma5 K = 1 - kappa*hopping (the Wilson operator up to the factor 2 kappa)."""
    kap = kappa_of_m(m0)
    return psi - kap * hopping(U, psi, antiperiodic_t)


def apply_K_sites(U, psi, m0, sites, antiperiodic_t=False):
    """(K psi)(x) at the listed sites only, x = (x, y, z, t) rows of ``sites``:
    the same formula evaluated from the 8 neighbours of each site (for spot checks
    of large lattices)."""
    kap = kappa_of_m(m0)
    lt, lz, ly, lx = psi.shape[:4]
    L = (lx, ly, lz, lt)
    out = []
    for (x, y, z, t) in np.asarray(sites):
        c = [int(x), int(y), int(z), int(t)]
        acc = np.zeros((4, 3), dtype=np.complex128)
        for mu in range(4):
            f = list(c)
            f[mu] = (c[mu] + 1) % L[mu]
            sf = -1.0 if (antiperiodic_t and mu == 3 and c[3] == L[3] - 1) else 1.0
            b = list(c)
            b[mu] = (c[mu] - 1) % L[mu]
            sb = -1.0 if (antiperiodic_t and mu == 3 and c[3] == 0) else 1.0
            pf = sf * psi[f[3], f[2], f[1], f[0]]
            pb = sb * psi[b[3], b[2], b[1], b[0]]
            Uf = U[c[3], c[2], c[1], c[0], mu]
            Ub = U[b[3], b[2], b[1], b[0], mu]
            acc += (I4 - GAMMA[mu]) @ (pf @ Uf.T)
            acc += (I4 + GAMMA[mu]) @ (pb @ np.conj(Ub))
        out.append(GAMMA5 @ (psi[c[3], c[2], c[1], c[0]] - kap * acc))
    return np.array(out)


def dense_operator(apply, site_shape):
    """Dense matrix of a linear map on spinors: column j = apply(e_j)."""
    n = int(np.prod(site_shape)) * 12
    eye = np.eye(n, dtype=np.complex128).reshape((n,) + tuple(site_shape) + (4, 3))
    cols = apply(eye)                                   # batched over the leading axis
    return cols.reshape(n, n).T.copy()


def dense_K(U, m0, antiperiodic_t=False):
    site_shape = U.shape[:4]
    return dense_operator(lambda v: apply_K(U, v, m0, antiperiodic_t), site_shape)


def sparse_K(U, m0, antiperiodic_t=False):
    """K of Sec. 1 (aK_xy) as a scipy CSR matrix on the flattened canonical spinor
    ordering (site, spin, colour), for the larger lattices where dense_K does not fit.

    Block row x holds gamma5 (1 x 1) at column block x, -kappa gamma5 (1 - gamma_mu) x U_mu(x)
    at x + mu and -kappa gamma5 (1 + gamma_mu) x U_mu(x - mu)^dag at x - mu, the t hops that
    cross the boundary negated when antiperiodic_t. The same formula as apply_K, assembled
    as explicit 12 x 12 (spin x colour) blocks instead of applied."""
    import scipy.sparse as sps
    lt, lz, ly, lx = U.shape[:4]
    V = lt * lz * ly * lx
    kap = kappa_of_m(m0)
    site = np.arange(V).reshape(lt, lz, ly, lx)
    Us = U.reshape(V, 4, 3, 3)
    tco = np.broadcast_to(np.arange(lt)[:, None, None, None], (lt, lz, ly, lx)).ravel()
    blocks = [np.broadcast_to(np.kron(GAMMA5, np.eye(3)), (V, 12, 12))]
    cols = [site.ravel()]
    for mu in range(4):
        ax = MU_AXIS[mu]
        fwd = np.roll(site, -1, axis=ax).ravel()      # x + mu
        bwd = np.roll(site, +1, axis=ax).ravel()      # x - mu
        sf = np.ones(V)
        sb = np.ones(V)
        if antiperiodic_t and mu == 3:
            sf[tco == lt - 1] = -1.0
            sb[tco == 0] = -1.0
        Pm = GAMMA5 @ (I4 - GAMMA[mu])
        Pp = GAMMA5 @ (I4 + GAMMA[mu])
        # (P x W)[(s, a), (t, b)] = P[s, t] W[a, b]
        Bf = np.einsum("st,xab->xsatb", Pm, Us[:, mu]).reshape(V, 12, 12)
        Bb = np.einsum("st,xba->xsatb", Pp, np.conj(Us[bwd, mu])).reshape(V, 12, 12)
        blocks += [-kap * sf[:, None, None] * Bf, -kap * sb[:, None, None] * Bb]
        cols += [fwd, bwd]
    data = np.stack(blocks, axis=1).reshape(-1, 12, 12)
    indices = np.stack(cols, axis=1).ravel()
    indptr = np.arange(0, 9 * V + 1, 9)
    M = sps.bsr_matrix((data, indices, indptr), shape=(12 * V, 12 * V)).tocsr()
    M.sum_duplicates()          # 2-site extents: x + mu and x - mu are one site
    M.eliminate_zeros()
    return M


def free_field_K_abs_spectrum(dims, m0, antiperiodic_t=False):
    """|lambda(K)| for U = 1, from the plane-wave closed form.

    With psi = e^{ipx} u, the hopping term gives sum_mu [2cos p_mu - 2i gamma_mu sin p_mu],
    so gamma5 K = 2 kappa [ b(p) + i gamma.s(p) ], b = sum_mu (1 - cos p_mu) - m0,
    s_mu = sin p_mu, hence |lambda| = 2 kappa sqrt(b^2 + |s|^2), 12-fold per momentum
    (4 spins x 3 colours; the sign splits 6/6).
    """
    lx, ly, lz, lt = dims
    kap = kappa_of_m(m0)
    ps = [2 * np.pi * np.arange(L) / L for L in (lx, ly, lz)]
    pt = 2 * np.pi * (np.arange(lt) + (0.5 if antiperiodic_t else 0.0)) / lt
    P = np.meshgrid(ps[0], ps[1], ps[2], pt, indexing="ij")
    b = sum(1 - np.cos(p) for p in P) - m0
    s2 = sum(np.sin(p) ** 2 for p in P)
    lam = 2 * kap * np.sqrt(b ** 2 + s2)
    return np.sort(np.repeat(lam.ravel(), 12))
