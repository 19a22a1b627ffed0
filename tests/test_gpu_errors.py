"""Failure reporting through the C ABI: a multi-shift CG that reaches its iteration
limit before the sign accuracy is met returns OVL_ENOCONV from every entry point that
applies the sign (sign, overlap apply, solve, gradient) instead of an inaccurate
result; the autograd wrapper refuses links other than the context's."""
import numpy as np
import pytest

import synth
from tests.gpu_util import lib, ctx

pytestmark = pytest.mark.gpu
DIMS = (4, 4, 4, 4)


def _capped(**kw):
    U = synth.gauge_links(DIMS, 0.3, 1001)
    return U, ctx(DIMS, U, n_poles=12, eps=1e-8, a=0.2, b=2.6, mscg_max=5, **kw)


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_sign_iteration_limit_is_an_error(prec):
    B = lib()
    U, c = _capped()
    v = synth.gaussian_source(DIMS, 3)
    out = np.zeros_like(v)
    with pytest.raises(B.OvlError) as e:
        c.sign_apply(v, out, eta=1e-8, prec=prec)
    assert e.value.status == B.OVL_ENOCONV
    assert "mscg_max" in str(e.value)
    with pytest.raises(B.OvlError) as e:
        c.apply(v, out, eta=1e-8, prec=prec)
    assert e.value.status == B.OVL_ENOCONV


def test_solve_and_gradient_pass_the_error_on():
    B = lib()
    U, c = _capped(mixed=0)
    b = synth.gaussian_source(DIMS, 4)
    x = np.zeros_like(b)
    with pytest.raises(B.OvlError) as e:
        c.solve(b, x, 1e-10)
    assert e.value.status == B.OVL_ENOCONV
    with pytest.raises(B.OvlError) as e:
        c.force(b, tol=1e-10)
    assert e.value.status == B.OVL_ENOCONV


def test_autograd_rejects_other_links():
    import torch
    from paper_1501_01855_gb300.autograd import overlap_action
    dims = (2, 2, 2, 2)
    U = synth.gauge_links(dims, 0.3, 41)
    phi = torch.from_numpy(synth.gaussian_source(dims, 42))
    c = ctx(dims, U, mu=0.05, n_poles=8, eps=1e-6, a=0.15, b=2.6, mixed=0)
    U2 = U.copy()
    U2[0, 0, 0, 0, 1] = synth.gauge_links((1, 1, 1, 1), 0.3, 7)[0, 0, 0, 0, 1]
    with pytest.raises(ValueError):
        overlap_action(torch.from_numpy(U2).requires_grad_(True), phi, c)
    S = overlap_action(torch.from_numpy(U.copy()).requires_grad_(True), phi, c)
    assert np.isfinite(S.item())


def test_gram_and_kernel_deflation_reject_bad_arguments():
    """Sizes, precisions and methods outside the documented ranges are OVL_EINVAL with the
    context left usable; a kernel deflation that cannot converge is OVL_ENOCONV and leaves
    the context undeflated (its original rational)."""
    import ctypes
    B = lib()
    U = synth.gauge_links(DIMS, 0.3, 1001)
    c = ctx(DIMS, U, n_poles=12, eps=1e-8, a=0.2, b=2.6)
    v = synth.gaussian_source(DIMS, 5, nvec=2)
    G = np.zeros(8)
    ptr = v.ctypes.data_as(ctypes.c_void_p)
    gp = G.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for na, nb, prec, method in ((0, 2, 0, 0), (2, 1025, 0, 0), (2, 2, 2, 0), (2, 2, 0, 2)):
        st = B.load().ovl_gram(c.h, ptr, na, ptr, nb, B.OVL_C128, 0, prec, 0, method, gp)
        assert st == B.OVL_EINVAL, (na, nb, prec, method, st)
    ms = ctypes.c_double()
    assert B.load().ovl_bench_gram(c.h, 2, 4, 4, 0, 1, ctypes.byref(ms)) == B.OVL_EINVAL
    for n_ev, n_poles in ((257, 0), (4, 65), (-1, 0)):
        with pytest.raises(B.OvlError) as e:
            c.kernel_deflate(n_ev, n_poles=n_poles)
        assert e.value.status == B.OVL_EINVAL
    om0, sg0, de0, a0, _ = c.zolotarev()
    with pytest.raises(B.OvlError) as e:
        c.kernel_deflate(6, tol=1e-14, max_iter=1)
    assert e.value.status == B.OVL_ENOCONV
    om1, sg1, de1, a1, _ = c.zolotarev()
    assert a1 == a0 and np.array_equal(om1, om0) and np.array_equal(sg1, sg0)
    # still usable
    assert np.allclose(c.gram(v, v), np.conj(v.reshape(2, -1)) @ v.reshape(2, -1).T, rtol=1e-12, atol=0)
    c.close()
