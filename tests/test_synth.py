"""The seeded input generators shared by the oracle tests, the GPU tests and the
benchmark: reproducible, of the stated layouts, and the links in SU(3)."""
import numpy as np

import synth


def test_gauge_links_are_su3_and_reproducible():
    dims = (4, 2, 2, 4)
    U = synth.gauge_links(dims, 0.3, 123)
    assert U.shape == (4, 2, 2, 4, 4, 3, 3)
    uu = np.einsum("...ij,...kj->...ik", U, np.conj(U))
    assert np.allclose(uu, np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)
    assert np.array_equal(U, synth.gauge_links(dims, 0.3, 123))
    assert not np.array_equal(U, synth.gauge_links(dims, 0.3, 124))
    # eps sets the distance from the identity
    near = synth.gauge_links(dims, 0.01, 5)
    assert np.abs(near - np.eye(3)).max() < 0.1


def test_sources_layouts():
    dims = (4, 2, 2, 4)
    g = synth.gaussian_source(dims, 7, nvec=3)
    assert g.shape == (3, 4, 2, 2, 4, 4, 3) and g.dtype == np.complex128
    assert np.array_equal(g[1], synth.gaussian_source(dims, 7, nvec=3)[1])
    p = synth.point_source(dims, 2, 1, site=(3, 1, 0, 2))
    assert p.sum() == 1.0 and p[2, 0, 1, 3, 2, 1] == 1.0
    z = synth.z2_source(dims, 9)
    assert set(np.unique(z.real)) <= {-1.0, 1.0} and np.all(z.imag == 0)
    u = synth.unit_links(dims)
    assert np.array_equal(u[0, 0, 0, 0, 2], np.eye(3))
