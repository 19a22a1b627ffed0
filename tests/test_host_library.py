"""CPU-side checks of liboverlap: the library loads, exports every symbol that
include/overlap.h declares, and its host-only numerics (Zolotarev coefficients
from its own elliptic-function code) agree with the oracle. No GPU calls."""
import os
import re

import numpy as np
import pytest

from oracle import zolotarev as zo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1501_01855_gb300 import build, binding
    build.build()
    return binding


def test_exports_every_declared_symbol():
    binding = _lib()
    lib = binding.load()
    hdr = open(os.path.join(ROOT, "include", "overlap.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b((?:ovl|overlap|eigsumr)_[a-z0-9_]+)\s*\(", hdr))
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(binding.exported_symbols()) == names


@pytest.mark.parametrize("n,a,b", [(1, 0.2, 2.5), (4, 0.1, 2.5), (16, 0.2136, 2.483), (24, 0.05, 2.54)])
def test_library_zolotarev_matches_oracle(n, a, b):
    binding = _lib()
    om, sg, de = binding.ovl_zolotarev_coeffs(n, a, b)
    o2, s2, d2 = zo.zolotarev(n, a, b)
    assert np.allclose(om, o2, rtol=1e-11, atol=0)
    assert np.allclose(sg, s2, rtol=1e-11, atol=0)
    assert abs(de - d2) <= 1e-6 * d2 + 5e-15


def test_library_rejects_bad_arguments():
    binding = _lib()
    with pytest.raises(binding.OvlError):
        binding.ovl_zolotarev_coeffs(0, 0.1, 1.0)
    with pytest.raises(binding.OvlError):
        binding.ovl_zolotarev_coeffs(4, 1.0, 0.5)


def test_binding_checks_output_buffers():
    """The binding refuses an output that is smaller than the input, of another dtype or
    on the other side of the bus, before any library call (so the library never writes
    past the end of a caller buffer)."""
    binding = _lib()
    x = np.zeros((2, 2, 2, 2, 4, 3), dtype=np.complex128)
    binding._io(None, x, np.zeros_like(x))
    with pytest.raises(ValueError):
        binding._io(None, x, np.zeros((1, 2, 2, 2, 4, 3), dtype=np.complex128))
    with pytest.raises(ValueError):
        binding._io(None, x, np.zeros_like(x, dtype=np.complex64))
    ro = np.zeros_like(x)
    ro.setflags(write=False)
    with pytest.raises(ValueError):
        binding._io(None, x, ro)
    import torch
    with pytest.raises(ValueError):
        binding._io(None, torch.zeros((2, 3), dtype=torch.complex128), torch.zeros((2, 2), dtype=torch.complex128))
