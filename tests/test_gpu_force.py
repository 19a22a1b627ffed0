"""Gauge-link gradient of S = phi^dag (D^dag D)^-1 phi through the C ABI against the
oracle's gradient (2^4 and a ragged antiperiodic lattice) and against central finite
differences of the library's own action on 8^4 along random Lie-algebra directions,
with the Zolotarev coefficients held fixed."""
import numpy as np
import pytest

import synth
from oracle import force, zolotarev as zo
from tests.gpu_util import ctx, rel, M0

pytestmark = pytest.mark.gpu
MU = 0.05


@pytest.mark.parametrize("dims,apt", [((2, 2, 2, 2), 0), ((4, 2, 2, 4), 1)])
def test_force_matches_oracle(dims, apt):
    U = synth.gauge_links(dims, 0.3, 31)
    phi = synth.gaussian_source(dims, 32)
    a, b = 0.15, 2.6
    c = ctx(dims, U, mu=MU, n_poles=8, eps=1e-6, a=a, b=b, mixed=0, bc_t=apt)
    G, S = c.force(phi, tol=1e-12)
    om, sg, _ = zo.zolotarev(8, a, b)
    Gref = force.gradient(U, phi, M0, MU, om, sg, tol=1e-13, antiperiodic_t=bool(apt))
    Sref, _ = force.action(U, phi, M0, MU, om, sg, tol=1e-13, antiperiodic_t=bool(apt))
    assert abs(S - Sref) <= 1e-9 * abs(Sref)
    assert rel(G, Gref) <= 1e-8


def test_force_finite_differences_8888():
    dims = (8, 8, 8, 8)
    U = synth.gauge_links(dims, 0.3, 1005)
    phi = synth.gaussian_source(dims, 2005)
    a, b = 0.2, 2.6
    kw = dict(mu=MU, n_poles=16, eps=1e-8, a=a, b=b)
    c = ctx(dims, U, **kw)
    G, S0 = c.force(phi, tol=1e-11)
    rng = np.random.Generator(np.random.PCG64(33))
    lam = synth._gell_mann()
    h = 1e-4
    for _ in range(4):
        X = np.einsum("...a,aij->...ij", rng.standard_normal(U.shape[:5] + (8,)), lam) * 0.5
        w, v = np.linalg.eigh(X)
        ex = lambda t: np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * t * w), np.conj(v))
        Sp = ctx(dims, ex(h) @ U, **kw).force(phi, tol=1e-11)[1]
        Sm = ctx(dims, ex(-h) @ U, **kw).force(phi, tol=1e-11)[1]
        fd = (Sp - Sm) / (2 * h)
        an = 2 * np.real(np.sum(np.conj(G) * (1j * X @ U)))
        # truncation O(h^2) plus the solve accuracy of S (1e-11 relative) over 2h
        assert abs(fd - an) <= 1e-5 * abs(an) + 10 * 1e-11 * abs(S0) / h, (fd, an)


def test_autograd_action_gradient_matches_oracle():
    """overlap_action (torch.autograd.Function over overlap_force): the action and U.grad
    against the oracle action and gradient (grad = 2 G in PyTorch's convention)."""
    import torch
    from paper_1501_01855_gb300.autograd import overlap_action
    dims = (2, 2, 2, 2)
    U = synth.gauge_links(dims, 0.3, 41)
    phi = synth.gaussian_source(dims, 42)
    a, b = 0.15, 2.6
    c = ctx(dims, U, mu=MU, n_poles=8, eps=1e-6, a=a, b=b, mixed=0)
    Ut = torch.from_numpy(U.copy()).requires_grad_(True)
    S = overlap_action(Ut, torch.from_numpy(phi), c, tol=1e-12)
    S.backward()
    om, sg, _ = zo.zolotarev(8, a, b)
    Sref, _ = force.action(U, phi, M0, MU, om, sg, tol=1e-13)
    Gref = force.gradient(U, phi, M0, MU, om, sg, tol=1e-13)
    assert abs(S.item() - Sref) <= 1e-9 * abs(Sref)
    assert rel(Ut.grad.numpy(), 2.0 * Gref) <= 1e-8
