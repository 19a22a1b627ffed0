"""GB300 (sm_103a) implementation of the deflated overlap-fermion inverter of
Cundy & Lee, "The eigSUMR inverter for overlap fermions" (arXiv:1501.01855).

The product is liboverlap.so (C ABI in include/overlap.h, CUDA sources in csrc/);
``binding`` is its thin ctypes binding and ``build`` compiles it with nvcc.
"""
__all__ = ["binding", "build"]
