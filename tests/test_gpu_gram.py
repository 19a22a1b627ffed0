"""Gram blocks G[i, j] = (A_i, [gamma5] B_j) through the C ABI (ovl_gram) against NumPy in
FP64 (and exact rational arithmetic where the claim is exactness).

The library's default Gram path (tensor cores; operands split into six balanced 7-bit
digits, exact BF16 products, exact FP32 sums over 512 reals, double-float and FP64 above)
claims FP64-level accuracy: each operand is represented to 2^-43 of its vector's
power-of-two scale, so an entry is within about 2^-42 sqrt(K) |A_i| |B_j| in the worst
case and near 1e-14 |A_i| |B_j| on random data. The tests hold it to 1e-12 |A_i| |B_j|
(the CUDA-core path with FP32 products misses that by five orders of magnitude, which the
last test shows), and to exactness where the sums are integers.
"""
from fractions import Fraction

import numpy as np
import pytest

from tests.gpu_util import lib

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)   # 3072 complex elements per vector: 12 exact-sum chunks of 512 reals


def _spinors(n, seed, dims=DIMS, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    shp = (n,) + tuple(reversed(dims)) + (4, 3)
    return (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)).astype(dtype)


def _g5(x):
    y = x.copy()
    y[..., 2:, :] *= -1   # chiral basis: gamma5 = diag(1, 1, -1, -1)
    return y


def _ref(A, B, g5):
    Bm = _g5(B) if g5 else B
    return np.conj(A.reshape(len(A), -1)) @ Bm.reshape(len(B), -1).T


def _ctx():
    from tests.gpu_util import ctx
    import synth
    return ctx(DIMS, synth.gauge_links(DIMS, 0.3, 7), a=0.2, b=2.6)


def _scale(A, B):
    na = np.linalg.norm(A.reshape(len(A), -1), axis=1)
    nb = np.linalg.norm(B.reshape(len(B), -1), axis=1)
    return np.outer(na, nb)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("g5", [0, 1])
def test_gram_tensor_cores_fp64_level(prec, g5):
    """70 x 70 (ragged tiles of 64) with per-vector scales from 1e-30 to 1e+30 and one zero
    vector; FP32 storage is compared with the FP32-rounded inputs in FP64."""
    Bn = lib()
    c = _ctx()
    A = _spinors(70, 11)
    B = _spinors(70, 12)
    A *= np.logspace(-30, 30, 70)[:, None, None, None, None, None, None]
    B *= np.logspace(20, -20, 70)[:, None, None, None, None, None, None]
    A[5] = 0
    p = Bn.OVL_PREC_F64 if prec == "f64" else Bn.OVL_PREC_F32
    if prec == "f32":
        A = A.astype(np.complex64).astype(np.complex128)
        B = B.astype(np.complex64).astype(np.complex128)
    G = c.gram(A, B, g5=g5, prec=p, method=0)
    c.close()
    ref = _ref(A, B, g5)
    err = np.abs(G - ref) / _scale(A, B)
    err[5] = np.abs(G[5])
    print("%s g5 %d: max |G - G_ref| / (|A_i| |B_j|) = %.3e" % (prec, g5, np.nanmax(err)))
    assert np.all(G[5] == 0)
    assert np.nanmax(err) <= 1e-12


def test_gram_integer_sums_exact():
    """Integer entries: every product and sum is an integer below 2^53, so G must equal the
    NumPy result exactly."""
    Bn = lib()
    c = _ctx()
    rng = np.random.default_rng(13)
    shp = (20,) + tuple(reversed(DIMS)) + (4, 3)
    A = (rng.integers(-1000, 1001, shp) + 1j * rng.integers(-1000, 1001, shp)).astype(np.complex128)
    B = (rng.integers(-1000, 1001, shp) + 1j * rng.integers(-1000, 1001, shp)).astype(np.complex128)
    G = c.gram(A, B, prec=Bn.OVL_PREC_F64)
    c.close()
    assert np.array_equal(G, _ref(A, B, 0))


def test_gram_worst_case_digits():
    """Every real equal to +-(1 - 2^-20): its leading digit is the largest the splitting
    produces (128), so the first group's FP32 sum reaches 2^23 in every chunk of 512 reals
    and the next ones come close to their 2^24 bound. Any rounding of those sums would show
    at 1e-8 relative; the result must be the exact rational value to 1e-14."""
    Bn = lib()
    c = _ctx()
    x = 1.0 - 2.0 ** -20
    A = np.full((2,) + tuple(reversed(DIMS)) + (4, 3), x + 1j * x)
    A[1] = -x + 1j * x
    G = c.gram(A, A, prec=Bn.OVL_PREC_F64)
    c.close()
    k = A[0].size
    xx = Fraction(x) * Fraction(x)
    exact = {(0, 0): (2 * k * xx, 0), (1, 1): (2 * k * xx, 0), (0, 1): (0, 2 * k * xx), (1, 0): (0, -2 * k * xx)}
    for (i, j), (re, im) in exact.items():
        want = complex(float(re), float(im))
        assert abs(G[i, j] - want) <= 1e-14 * abs(want), (i, j, G[i, j], want)


def test_gram_cuda_core_path_agrees_and_is_fp32_level():
    """method 1 (CUDA cores, FP32 products) against the same reference: FP32 level only,
    which is why the tensor-core path is the default."""
    Bn = lib()
    c = _ctx()
    A = _spinors(16, 21)
    B = _spinors(9, 22)
    G0 = c.gram(A, B, g5=1, method=0)
    G1 = c.gram(A, B, g5=1, method=1)
    c.close()
    ref = _ref(A, B, 1)
    s = _scale(A, B)
    e0 = np.max(np.abs(G0 - ref) / s)
    e1 = np.max(np.abs(G1 - ref) / s)
    print("tensor cores %.3e, CUDA cores (FP32 products) %.3e" % (e0, e1))
    assert e0 <= 1e-12
    assert 1e-12 < e1 <= 1e-5


def test_gram_device_buffers_and_large_lattice():
    """Device tensors in, on 8^3 x 16 (98304 complex elements per vector, 384 chunks split
    over the SMs) with 130 x 40 vectors: three A tiles against one ragged B tile."""
    import torch
    Bn = lib()
    from tests.gpu_util import ctx
    import synth
    dims = (8, 8, 8, 16)
    c = ctx(dims, synth.gauge_links(dims, 0.3, 8), a=0.2, b=2.6)
    A = _spinors(130, 31, dims)
    B = _spinors(40, 32, dims)
    G = c.gram(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec=Bn.OVL_PREC_F64)
    c.close()
    err = np.max(np.abs(G - _ref(A, B, 0)) / _scale(A, B))
    print("8^3x16, 130 x 40: %.3e" % err)
    assert err <= 1e-12
