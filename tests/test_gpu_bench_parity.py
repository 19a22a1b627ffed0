"""The benchmarked calls against the oracle at sizes the oracle finishes in seconds.

* The overlap apply exactly as bench.py issues it (16 Gaussian vectors in one call,
  20 Zolotarev poles, eta = 1e-10, double-float stored-basis Lanczos sign, cached step
  graphs, autotuned Wilson launch shape), on 8^4 and 8^3 x 16 (and the multi-shift CG form
  on 8^4), compared element by element with
  the oracle's per-pole CG (its own Zolotarev coefficients for the same [a, b]) on
  vectors 0, 7 and 15; every system of the batch is independent arithmetic, which
  test_sign_sub_batches_match_one_batch pins bit for bit.
* Batched, deflated, multi-mass solves shaped like the 16^3 x 32 and 24^3 x 48
  configurations (12 point sources x 3 masses in one call, an eigSUMR space shared by
  the masses, 24 poles) on 8^4, with relSUMR and with relCG as middle solver, each
  checked with the oracle's true residual ||b - D_oracle x|| / ||b|| <= 1e-10 on
  sources 0, 5 and 11 of every mass (the oracle's rational is the library's: same
  n and [a, b], Sec. 3).
"""
import os

import numpy as np
import pytest

import synth
from oracle import overlap, zolotarev as zo
from tests.gpu_util import lib, ctx, M0

pytestmark = pytest.mark.gpu

A, B = 0.2, 2.6
WORKERS = max(1, min(16, len(os.sched_getaffinity(0))))


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("dims,method", [((8, 8, 8, 8), 0), ((8, 8, 8, 16), 0), ((8, 8, 8, 8), 1)])
def test_bench_apply_matches_oracle(dims, method):
    """method 0: the default stored-basis Lanczos sign (the benchmarked path); 1: the
    multi-shift CG form."""
    import torch
    Bn = lib()
    mu, npoles, eta = 0.05, 20, 1e-10
    U = synth.gauge_links(dims, 0.3, 1002)
    vecs = synth.gaussian_source(dims, 2002, nvec=16)
    c = ctx(dims, U, mu=mu, n_poles=npoles, eps=1e-10, a=A, b=B, sign_method=method)   # graphs on, autotuned shape
    dv = torch.from_numpy(vecs).cuda()
    dout = torch.empty_like(dv)
    c.apply(dv, dout, eta=eta, prec=Bn.OVL_PREC_F64E)
    c.apply(dv, dout, eta=eta, prec=Bn.OVL_PREC_F64E)   # the second call replays cached graphs
    got = dout.cpu().numpy()
    c.close()
    om, sg, de = zo.zolotarev(npoles, A, B)
    pick = [0, 7, 15]
    ref = overlap.overlap_apply_many(U, vecs[pick], M0, mu, om, sg, tol=1e-14, workers=WORKERS)
    for k, j in enumerate(pick):
        err = _rel(got[j], ref[k])
        pointwise = np.abs(got[j] - ref[k]).max() / np.abs(ref[k]).max()
        print("%s method %d vector %d: relative error %.3e, max pointwise %.3e" % (dims, method, j, err, pointwise))
        assert err <= 1e-9
        assert pointwise <= 1e-9


def _c4_shaped_setup(solver):
    dims = (8, 8, 8, 8)
    U = synth.gauge_links(dims, 0.3, 1004)
    srcs = np.stack([synth.point_source(dims, s, col) for s in range(4) for col in range(3)])
    mus = [0.01, 0.02, 0.04]
    c = ctx(dims, U, mu=mus[0], n_poles=24, eps=1e-10, a=A, b=B, solver=solver)
    return dims, U, srcs, mus, c


@pytest.mark.parametrize("solver", [0, 1])
def test_multimass_deflated_batch_true_residual(solver):
    dims, U, srcs, mus, c = _c4_shaped_setup(solver)
    defl = None
    for k in range(2):
        b0 = synth.gaussian_source(dims, 2004 + k)
        x0 = np.zeros_like(b0)
        defl, _ = c.eigsumr_accumulate(b0, x0, 1e-10, 16, 40, defl=defl)
    xs = np.zeros((len(mus) * len(srcs),) + srcs.shape[1:], dtype=np.complex128)
    infos = c.solve(srcs, xs, 1e-10, mus=mus, defl=defl)
    defl.close()
    c.close()
    assert all(i["converged"] == 1 for i in infos)
    assert max(i["true_residual"] for i in infos) <= 1e-10
    om, sg, _ = zo.zolotarev(24, A, B)
    pick = [(m, j) for m in range(3) for j in (0, 5, 11)]
    X = np.stack([xs[m * 12 + j] for m, j in pick])
    DX = overlap.overlap_apply_many(U, X, M0, [mus[m] for m, _ in pick], om, sg, tol=1e-14, workers=WORKERS)
    for k, (m, j) in enumerate(pick):
        tr = np.linalg.norm(srcs[j] - DX[k]) / np.linalg.norm(srcs[j])
        print("solver %d mu %.2f source %d: oracle true residual %.3e (library %.3e)"
              % (solver, mus[m], j, tr, infos[m * 12 + j]["true_residual"]))
        assert tr <= 1e-10
