"""Overlap solves through the C ABI against the oracle: GMRESR(relSUMR) and
GMRESR(relCG), mixed precision and plain FP64, to a relative true residual of
1e-10 measured with the oracle's dense operator (config 1: 4^4, m0 = 1.4,
mu = 0.05, 16 poles, eps 1e-10), several sources and masses in one batch."""
import numpy as np
import pytest

import synth
from oracle import overlap
from tests.gpu_util import lib, ctx, rel, dense_4444

pytestmark = pytest.mark.gpu
DIMS = (4, 4, 4, 4)


def _check(U, S, x, b, mu, tol):
    D = overlap.dense_overlap(S, mu, 256)
    r = b.ravel() - D @ x.ravel()
    tr = np.linalg.norm(r) / np.linalg.norm(b)
    xs = np.linalg.solve(D, b.ravel())
    err = np.linalg.norm(x.ravel() - xs) / np.linalg.norm(xs)
    return tr, err


@pytest.mark.parametrize("mixed,solver,emul", [(1, 0, 0), (0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 0, 1)])
def test_config1_solve(mixed, solver, emul):
    U, Kd, S, w = dense_4444()
    c = ctx(DIMS, U, mu=0.05, n_poles=16, mixed=mixed, solver=solver, emulate_fp64=emul)
    b = synth.gaussian_source(DIMS, 2001)
    x = np.zeros_like(b)
    info = c.solve(b, x, 1e-10)
    tr, err = _check(U, S, x, b, 0.05, 1e-10)
    print("mixed=%d solver=%d true residual %.3e, error %.3e, info %s" % (mixed, solver, tr, err, info[0]))
    assert tr <= 1e-10
    assert err <= 20 * 1e-10
    assert info[0]["converged"] == 1
    assert info[0]["true_residual"] <= 1e-10


def test_batched_sources_and_masses():
    U, Kd, S, w = dense_4444()
    c = ctx(DIMS, U, mu=0.05, n_poles=16)
    b = np.stack([synth.point_source(DIMS, s, col) for s, col in ((0, 0), (3, 2))])
    mus = [0.02, 0.1]
    x = np.zeros((2,) + b.shape, dtype=np.complex128)
    info = c.solve(b, x, 1e-10, mus=mus)
    for k, mu in enumerate(mus):
        for j in range(2):
            tr, err = _check(U, S, x[k, j], b[j], mu, 1e-10)
            assert tr <= 1e-10, (k, j, tr)
    # lock-step batching gives the per-system answer
    x1 = np.zeros_like(b[1])
    c.solve(np.ascontiguousarray(b[1]), x1, 1e-10, mus=[0.1])
    assert rel(x[1, 1], x1) <= 1e-8


def test_multimass_shared_basis_matches_independent():
    """Three masses of two sources: with the first middle solve sharing one SUMR basis per
    source (multimass = 1, the default) every solution meets the oracle's true residual,
    agrees with the independent per-system solves (multimass = 0) to the solve accuracy,
    and the batch needs fewer Wilson applications."""
    U, Kd, S, w = dense_4444()
    b = np.stack([synth.point_source(DIMS, 0, 1), synth.gaussian_source(DIMS, 2003)])
    mus = [0.02, 0.05, 0.2]
    out = {}
    for mm in (1, 0):
        c = ctx(DIMS, U, mu=0.05, n_poles=16, multimass=mm)
        x = np.zeros((3,) + b.shape, dtype=np.complex128)
        info = c.solve(b, x, 1e-10, mus=mus)
        for k, mu in enumerate(mus):
            for j in range(2):
                tr, err = _check(U, S, x[k, j], b[j], mu, 1e-10)
                assert tr <= 1e-10, (mm, k, j, tr)
        out[mm] = (x, sum(i["wilson_calls"] for i in info))
    for k, mu in enumerate(mus):
        for j in range(2):
            assert rel(out[1][0][k, j], out[0][0][k, j]) <= 2e-8 / mu
    print("Wilson calls: shared basis %d, independent %d" % (out[1][1], out[0][1]))
    assert out[1][1] < out[0][1]
