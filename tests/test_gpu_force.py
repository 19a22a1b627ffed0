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


@pytest.mark.parametrize("dims,apt,mixed", [((2, 2, 2, 2), 0, 0), ((4, 2, 2, 4), 1, 0), ((2, 2, 2, 2), 0, 1)])
def test_force_matches_oracle(dims, apt, mixed):
    """mixed = 1: the FP32 adjoint (FP32 outer products, FP64 accumulation), held to the
    FP32 level of its products."""
    U = synth.gauge_links(dims, 0.3, 31)
    phi = synth.gaussian_source(dims, 32)
    a, b = 0.15, 2.6
    c = ctx(dims, U, mu=MU, n_poles=8, eps=1e-6, a=a, b=b, mixed=mixed, bc_t=apt)
    G, S = c.force(phi, tol=1e-12)
    om, sg, _ = zo.zolotarev(8, a, b)
    Gref = force.gradient(U, phi, M0, MU, om, sg, tol=1e-13, antiperiodic_t=bool(apt))
    Sref, _ = force.action(U, phi, M0, MU, om, sg, tol=1e-13, antiperiodic_t=bool(apt))
    err = rel(G, Gref)
    print("dims %s mixed %d: gradient %.3e, action %.3e" % (dims, mixed, err, abs(S - Sref) / abs(Sref)))
    assert abs(S - Sref) <= 1e-9 * abs(Sref)
    assert err <= (1e-8 if mixed == 0 else 1e-6)


def test_force_finite_differences_8888():
    """The FP32 adjoint (mixed = 1: FP32 outer products, FP64 accumulation) against central
    differences of the action on 32 random Lie-algebra directions on 8^4 (16 poles)."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_links(dims, 0.3, 1005)
    phi = synth.gaussian_source(dims, 2005)
    a, b = 0.2, 2.6
    kw = dict(mu=MU, n_poles=16, eps=1e-8, a=a, b=b)
    c = ctx(dims, U, mixed=1, **kw)
    G, S0 = c.force(phi, tol=1e-11)
    rng = np.random.Generator(np.random.PCG64(33))
    lam = synth._gell_mann()
    h = 1e-4
    for _ in range(32):
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


@pytest.mark.parametrize("mixed", [0, 1])
def test_force_4444_matches_dense_oracle(mixed):
    """4^4, 16 poles: the gradient in FP64 (mixed = 0) and with the FP32 adjoint kernel
    (mixed = 1: FP32 outer products, FP64 accumulation) against the oracle's gradient
    (same formula, dense K); the FP32 one to FP32 rounding of the outer products."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_links(dims, 0.3, 51)
    phi = synth.gaussian_source(dims, 52)
    a, b = 0.2, 2.6
    c = ctx(dims, U, mu=MU, n_poles=16, eps=1e-6, a=a, b=b, mixed=mixed)
    G, S = c.force(phi, tol=1e-12)
    om, sg, _ = zo.zolotarev(16, a, b)
    Gref, Sref = force.gradient_dense(U, phi, M0, MU, om, sg)
    err = rel(G, Gref)
    print("mixed %d: gradient error %.3e, action error %.3e" % (mixed, err, abs(S - Sref) / abs(Sref)))
    assert abs(S - Sref) <= 1e-9 * abs(Sref)
    assert err <= (1e-8 if mixed == 0 else 2e-6)


def test_force_pole_groups_match_all_at_once():
    """Shifted solutions recomputed in groups of 3 poles (16 poles: five full groups and
    one of one) give the gradient of the all-at-once path."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_links(dims, 0.3, 53)
    phi = synth.gaussian_source(dims, 54)
    kw = dict(mu=MU, n_poles=16, eps=1e-6, a=0.2, b=2.6, mixed=0)
    G1, S1 = ctx(dims, U, force_pole_group=0, **kw).force(phi, tol=1e-12)
    G2, S2 = ctx(dims, U, force_pole_group=3, **kw).force(phi, tol=1e-12)
    assert abs(S1 - S2) <= 1e-12 * abs(S1)
    assert rel(G2, G1) <= 1e-9
