"""Parity of the Zolotarev sign function (multi-shift CG, Sec. 3) and of the
overlap operator D(mu) (Sec. 1) through the C ABI against the oracle (per-pole
plain CG with the oracle's own Zolotarev coefficients for the same [a, b], and
the dense spectral sign on 4^4), with the error of the FP32 / FP16 paths stated."""
import numpy as np
import pytest

import synth
from oracle import wilson, overlap, zolotarev as zo
from tests.gpu_util import lib, ctx, rel, dense_4444, M0

pytestmark = pytest.mark.gpu


def _ab(w):
    return 0.95 * np.min(np.abs(w)), 1.05 * np.max(np.abs(w))


@pytest.mark.parametrize("prec,method,cap", [(0, 0, 0), (3, 0, 0), (0, 1, 0), (3, 1, 0), (3, 2, 20), (0, 2, 9)])
def test_sign_fp64_matches_per_pole_oracle(prec, method, cap):
    """method 0: stored-basis Lanczos (cap 0: one cycle), 1: multi-shift CG, 2: Lanczos
    restarted every cap steps (several cycles)."""
    U, Kd, S, w = dense_4444()
    a, b = _ab(w)
    c = ctx((4, 4, 4, 4), U, a=a, b=b, n_poles=16, sign_method=method, lanczos_cap=cap)
    om, sg, de = zo.zolotarev(16, a, b)
    v = synth.gaussian_source((4, 4, 4, 4), 2001, nvec=2)
    out = np.zeros_like(v)
    c.sign_apply(v, out, eta=1e-11, prec=prec)
    for j in range(2):
        ref = overlap.zolotarev_sign_apply(U, v[j], M0, om, sg, tol=1e-14)
        assert rel(out[j], ref) <= 1e-9
        # and the spectral sign: the Zolotarev error is below 1e-10 here
        exact = (S @ v[j].ravel()).reshape(v[j].shape)
        assert rel(out[j], exact) <= 2e-10


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("prec,eta,bound", [(1, 1e-5, 2e-5), (2, 1e-2, 2e-2), (0, 1e-6, 2e-6)])
def test_sign_relaxed_accuracy(prec, eta, bound, method):
    U, Kd, S, w = dense_4444()
    a, b = _ab(w)
    c = ctx((4, 4, 4, 4), U, a=a, b=b, n_poles=16, sign_method=method)
    v = synth.gaussian_source((4, 4, 4, 4), 7)
    out = np.zeros_like(v)
    c.sign_apply(v, out, eta=eta, prec=prec)
    exact = (S @ v.ravel()).reshape(v.shape)
    err = rel(out, exact)
    print("sign prec=%d eta=%g method=%d error=%.3e" % (prec, eta, method, err))
    assert err <= bound


def test_sign_fp16_repeated_calls_keep_accuracy():
    """FP16 storage, stored-basis Lanczos, several calls on one context: the cycle length
    changes between calls (the first is sized from the CG bound, later ones from the steps
    seen), and with it the offset of the per-site scales inside the pooled basis; every
    call must still meet its accuracy (cached step graphs included)."""
    U, Kd, S, w = dense_4444()
    a, b = _ab(w)
    c = ctx((4, 4, 4, 4), U, a=a, b=b, n_poles=16, sign_method=0)
    v = synth.gaussian_source((4, 4, 4, 4), 7, nvec=2)
    exact = np.stack([(S @ v[j].ravel()).reshape(v[j].shape) for j in range(2)])
    for eta in (1e-2, 1e-2, 3e-3, 1e-2, 3e-3):
        out = np.zeros_like(v)
        c.sign_apply(v, out, eta=eta, prec=2)
        err = rel(out, exact)
        print("FP16 eta %g: error %.3e" % (eta, err))
        assert err <= 2 * eta
    c.close()


@pytest.mark.parametrize("mu,prec", [(0.05, 0), (0.3, 0), (0.05, 3)])
def test_overlap_apply_matches_dense(mu, prec):
    U, Kd, S, w = dense_4444()
    c = ctx((4, 4, 4, 4), U, mu=mu, n_poles=16)   # bounds from the library's Lanczos estimate
    D = overlap.dense_overlap(S, mu, 256)
    v = synth.gaussian_source((4, 4, 4, 4), 11, nvec=3)
    out = np.zeros_like(v)
    c.apply(v, out, mu=mu, eta=1e-11, prec=prec)
    hout = np.zeros_like(v)
    c.apply(v, hout, mu=mu, eta=1e-11, prec=prec, hermitian=True)
    for j in range(3):
        ref = (D @ v[j].ravel()).reshape(v[j].shape)
        assert rel(out[j], ref) <= 1e-9
        assert rel(hout[j], wilson.apply_gamma5(ref)) <= 1e-9


def test_overlap_apply_full_size_properties():
    """16^3x32: sign(K)^2 v = v and [sign(K), K] = 0 on sampled sites, FP64 and FP32."""
    dims = (16, 16, 16, 32)
    U = synth.gauge_links(dims, 0.3, 1002)
    c = ctx(dims, U, n_poles=20)
    om, sg, de, a, b = c.zolotarev()
    assert de <= 1e-10
    v = synth.gaussian_source(dims, 2002)
    s1 = np.zeros_like(v)
    s2 = np.zeros_like(v)
    c.sign_apply(v, s1, eta=1e-10, prec=0)
    c.sign_apply(s1, s2, eta=1e-10, prec=0)
    assert rel(s2, v) <= 5e-9
    Kv = np.zeros_like(v)
    c.wilson_apply(v, Kv, 0)
    sKv = np.zeros_like(v)
    c.sign_apply(Kv, sKv, eta=1e-10, prec=0)
    rng = np.random.default_rng(3)
    sites = np.stack([rng.integers(0, d, 32) for d in dims], axis=1)
    Ks = wilson.apply_K_sites(U, s1, M0, sites)
    got = np.array([sKv[t, z, y, x] for (x, y, z, t) in sites])
    assert rel(got, Ks) <= 5e-9
    e1 = np.zeros_like(v)
    c.sign_apply(v, e1, eta=1e-10, prec=3)
    print("16^3x32 double-float sign at eta=1e-10: difference to FP64 %.3e" % rel(e1, s1))
    assert rel(e1, s1) <= 5e-10
    f1 = np.zeros_like(v)
    c.sign_apply(v, f1, eta=1e-5, prec=1)
    print("16^3x32 FP32 sign at eta=1e-5: error vs FP64 %.3e" % rel(f1, s1))
    assert rel(f1, s1) <= 2e-5


def test_graph_replay_matches_stream_launches():
    """The multi-shift CG iterations replayed as CUDA graphs give bit-identical results to
    the same kernels launched one by one (fixed-order reductions, same launch shapes; the
    launch shape is fixed so that the autotuner's timing cannot pick different ones)."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_links(dims, 0.3, 1011)
    v = synth.gaussian_source(dims, 2011, nvec=3)
    outs = []
    for g in (0, 1):
        c = ctx(dims, U, n_poles=16, eps=1e-10, a=0.2, b=2.6, use_graphs=g, wilson_variant=0)
        o = np.zeros_like(v)
        c.apply(v, o, eta=1e-10)
        c.apply(v, o, eta=1e-10)   # second call replays the cached graph
        outs.append(o)
        c.close()
    assert np.array_equal(outs[0], outs[1])


def test_pinned_host_buffers_match_pageable():
    """Page-locked host buffers take the direct DMA path; the result is bit-identical
    to the pageable path through the staging buffer."""
    import torch
    dims = (8, 8, 8, 8)
    U = synth.gauge_links(dims, 0.3, 1031)
    v = synth.gaussian_source(dims, 2031, nvec=2)
    c = ctx(dims, U, n_poles=16, eps=1e-10, a=0.2, b=2.6)
    o1 = np.zeros_like(v)
    c.apply(v, o1, eta=1e-10)
    vp = torch.from_numpy(v).pin_memory()
    op = torch.zeros(v.shape, dtype=torch.complex128).pin_memory()
    c.apply(vp.numpy(), op.numpy(), eta=1e-10)
    assert np.array_equal(op.numpy(), o1)


def test_sign_sub_batches_match_one_batch():
    """Requests larger than the batch size run as consecutive multi-shift sub-batches;
    every system's arithmetic is independent of its batch, so the result is identical."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_links(dims, 0.3, 1041)
    v = synth.gaussian_source(dims, 2041, nvec=5)
    outs = []
    for bm in (36, 2):
        c = ctx(dims, U, n_poles=16, eps=1e-10, a=0.2, b=2.6, batch_max=bm, wilson_variant=0)
        o = np.zeros_like(v)
        c.sign_apply(v, o, eta=1e-10, prec=3)
        outs.append(o)
        c.close()
    assert np.array_equal(outs[0], outs[1])
