"""The allocation-free Wilson entry point (static device scratch) against the
ordinary one, through the C ABI, on two calls in a row; and its size limit.
Collected last so that a run stopping at the first failure has run everything else."""
import numpy as np
import pytest

import synth
from tests.gpu_util import ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6), (2, 4e-3)])
def test_noalloc_matches_wilson_apply_twice(prec, tol):
    import torch
    dims = (8, 8, 8, 8)
    U = synth.gauge_links(dims, 0.3, 1001)
    c = ctx(dims, U, a=0.1, b=2.6)
    for call, seed in enumerate((11, 12)):
        psi = torch.from_numpy(synth.gaussian_source(dims, seed, nvec=3)).cuda()
        ref = torch.zeros_like(psi)
        out = torch.full_like(psi, complex(float("nan"), 0.0))
        c.wilson_apply(psi, ref, prec)
        c.wilson_apply_noalloc(psi, out, prec)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        err = np.linalg.norm(o - r) / np.linalg.norm(r)
        assert np.all(np.isfinite(o)), call
        assert err <= tol, (call, err)


def test_noalloc_rejects_oversize_request():
    import torch
    from tests.gpu_util import lib
    dims = (16, 16, 16, 32)
    U = synth.unit_links(dims)
    c = ctx(dims, U, a=0.1, b=2.6)
    psi = torch.zeros((2,) + synth.lattice_shape(dims) + (4, 3), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(psi)
    with pytest.raises(lib().OvlError):
        c.wilson_apply_noalloc(psi, out, 0)          # 2 x 131072 sites in FP64 exceeds 48 MiB
    c.wilson_apply_noalloc(psi[:1].contiguous(), out[:1].contiguous(), 0)   # exactly at the limit
