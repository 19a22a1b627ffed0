"""Parity of the Wilson kernel K (Sec. 1) through the C ABI against the oracle:
FP64 / FP32 / FP16-storage kernels, periodic and antiperiodic t, ragged site
counts, multi-system launches, device and host buffers, and sampled sites of the
full-size lattices in the launch configuration the benchmark times."""
import numpy as np
import pytest

import synth
from oracle import wilson, overlap
from tests.gpu_util import lib, ctx, rel, M0

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-6, 2: 4e-3, 3: 2e-13}


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 2, 4, 6), (2, 2, 2, 2), (8, 8, 8, 4)])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("apt", [0, 1])
def test_wilson_matches_oracle(dims, prec, apt):
    U = synth.gauge_links(dims, 0.3, 1001)
    c = ctx(dims, U, a=0.1, b=2.6, bc_t=apt)
    psi = synth.gaussian_source(dims, 2001, nvec=3)
    out = np.zeros_like(psi)
    c.wilson_apply(psi, out, prec)
    for j in range(3):
        ref = wilson.apply_K(U, psi[j], M0, bool(apt))
        assert rel(out[j], ref) <= TOL[prec]


def test_wilson_device_buffers_and_batch_consistency():
    import torch
    dims = (4, 4, 4, 8)
    U = synth.gauge_links(dims, 0.3, 5)
    c = ctx(dims, U, a=0.1, b=2.6)
    psi = synth.gaussian_source(dims, 6, nvec=5)
    dpsi = torch.from_numpy(psi).cuda()
    dout = torch.zeros_like(dpsi)
    c.wilson_apply(dpsi, dout, 0)
    single = np.zeros_like(psi[0])
    c.wilson_apply(np.ascontiguousarray(psi[3]), single, 0)
    got = dout.cpu().numpy()
    assert np.array_equal(got[3], single)
    assert rel(got[1], wilson.apply_K(U, psi[1], M0)) <= 1e-13


@pytest.mark.parametrize("dims", [(16, 16, 16, 32), (24, 24, 24, 48)])
def test_wilson_full_size_sampled(dims):
    U = synth.gauge_links(dims, 0.3, 1002)
    c = ctx(dims, U, a=0.1, b=2.6)
    psi = synth.gaussian_source(dims, 2002)
    rng = np.random.default_rng(1)
    sites = np.stack([rng.integers(0, d, 64) for d in dims], axis=1)
    sites[0] = (dims[0] - 1, dims[1] - 1, dims[2] - 1, dims[3] - 1)
    sites[1] = (0, 0, 0, 0)
    ref = wilson.apply_K_sites(U, psi, M0, sites)
    for prec in (0, 1, 3):
        out = np.zeros_like(psi)
        c.wilson_apply(psi, out, prec)
        got = np.array([out[t, z, y, x] for (x, y, z, t) in sites])
        assert rel(got, ref) <= TOL[prec]
    # a property at any size: K is Hermitian, (a, K b) = (K a, b)
    b = synth.gaussian_source(dims, 2003)
    Kb = np.zeros_like(b)
    Kpsi = np.zeros_like(b)
    c.wilson_apply(b, Kb, 0)
    c.wilson_apply(psi, Kpsi, 0)
    l, r = np.vdot(psi, Kb), np.vdot(Kpsi, b)
    assert abs(l - r) <= 1e-12 * abs(l)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_wilson_launch_variants(variant, prec):
    """Every launch shape the autotuner can pick (thread per site, direction split, 4D
    tiles, lane pairs for double-float) gives K to the precision's tolerance, on a lattice
    that divides into tiles (two tiles in t) with antiperiodic t, for several systems at
    once."""
    dims = (8, 4, 8, 4)
    U = synth.gauge_links(dims, 0.3, 1021)
    c = ctx(dims, U, a=0.1, b=2.6, bc_t=1, wilson_variant=variant)
    assert c.wilson_tuning(prec)[0] == (variant if variant != 3 or prec == 3 else 0)
    psi = synth.gaussian_source(dims, 2021, nvec=5)
    out = np.zeros_like(psi)
    c.wilson_apply(psi, out, prec)
    for j in range(5):
        assert rel(out[j], wilson.apply_K(U, psi[j], M0, True)) <= TOL[prec]


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_sign_with_launch_variants(variant, method):
    """The sign function reads its scalars from the Wilson kernel's partial sums; with every
    launch shape, and with the stored-basis Lanczos (method 0) and the multi-shift CG
    (method 1), it matches the oracle's per-pole CG for the same rational."""
    from oracle import zolotarev as zo
    dims = (8, 4, 8, 4)
    U = synth.gauge_links(dims, 0.3, 1022)
    v = synth.gaussian_source(dims, 2022, nvec=2)
    om, sg, _ = zo.zolotarev(16, 0.2, 2.6)
    ref = [overlap.zolotarev_sign_apply(U, v[j], M0, om, sg, tol=1e-14) for j in range(2)]
    c = ctx(dims, U, n_poles=16, a=0.2, b=2.6, wilson_variant=variant, sign_method=method)
    for prec in (0, 3):
        out = np.zeros_like(v)
        c.sign_apply(v, out, eta=1e-11, prec=prec)
        for j in range(2):
            assert rel(out[j], ref[j]) <= 1e-10
