"""Seeded synthetic inputs for the overlap hot path: gauge links and sources.

This module only draws random numbers and builds SU(3) matrices; it holds none
of the overlap method's arithmetic. Both the oracle and the CUDA path take their
inputs from here, so that they see bit-identical data.

Canonical host layouts (C order, complex128):
  spinor  [Lt][Lz][Ly][Lx][spin 4][colour 3]
  links   [Lt][Lz][Ly][Lx][mu 4][row 3][col 3],   mu = 0,1,2,3 -> x,y,z,t
so that site = ((t*Lz + z)*Ly + y)*Lx + x.

The paper's gauge ensemble (an 8^3x32 dynamical overlap ensemble, Sec. 6) is
not available; smooth random SU(3) fields stand in for it:
U = proj_SU3(exp(i*eps*H)), H = sum_a h_a lambda_a / 2, h_a ~ N(0,1).
"""
import numpy as np

__all__ = ["lattice_shape", "gauge_links", "unit_links", "gaussian_source",
           "point_source", "z2_source", "random_su3_field", "project_su3"]


def lattice_shape(dims):
    """dims = (Lx, Ly, Lz, Lt) -> numpy site shape (Lt, Lz, Ly, Lx)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def _gell_mann():
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j; lam[1][1, 0] = 1j
    lam[2][0, 0] = 1; lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j; lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j; lam[6][2, 1] = 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam


def project_su3(m):
    """Gram-Schmidt on rows 1-2, then row3 = conj(row1 x row2). Works on (..., 3, 3)."""
    m = np.array(m, dtype=np.complex128, copy=True)
    r1 = m[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = m[..., 1, :]
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


def _expi_hermitian(h):
    """exp(i*h) for a stack of Hermitian 3x3 matrices, by eigendecomposition."""
    w, v = np.linalg.eigh(h)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def random_su3_field(shape, eps, rng):
    """proj_SU3(exp(i*eps*H)) with H = sum_a h_a lambda_a/2, h drawn in C order over shape."""
    h = rng.standard_normal(tuple(shape) + (8,))
    lam = _gell_mann()
    H = np.einsum("...a,aij->...ij", h, lam) * 0.5
    return project_su3(_expi_hermitian(eps * H))


def gauge_links(dims, eps=0.3, seed=1000):
    """Smooth random SU(3) links, shape (Lt,Lz,Ly,Lx,4,3,3), complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return random_su3_field(lattice_shape(dims) + (4,), eps, rng)


def unit_links(dims):
    """Free field U = 1."""
    u = np.zeros(lattice_shape(dims) + (4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1
    return u


def gaussian_source(dims, seed=2000, nvec=None):
    """Gaussian spinor(s): re, im ~ N(0,1) per component. nvec adds a leading axis."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = lattice_shape(dims) + (4, 3)
    if nvec is not None:
        shape = (int(nvec),) + shape
    z = rng.standard_normal(shape + (2,))
    return z[..., 0] + 1j * z[..., 1]


def point_source(dims, spin, colour, site=(0, 0, 0, 0)):
    """delta_{x,site} delta_{s,spin} delta_{c,colour}; site = (x,y,z,t)."""
    v = np.zeros(lattice_shape(dims) + (4, 3), dtype=np.complex128)
    x, y, z, t = site
    v[t, z, y, x, spin, colour] = 1.0
    return v


def z2_source(dims, seed=2000):
    """Each component +-1 with equal probability (the paper's source type, Sec. 6)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = rng.integers(0, 2, size=lattice_shape(dims) + (4, 3))
    return (2.0 * s - 1.0).astype(np.complex128)
