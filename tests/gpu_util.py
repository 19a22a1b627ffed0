"""Shared set-up of the GPU parity tests (test infrastructure)."""
import functools

import numpy as np

import synth
from oracle import wilson, overlap, zolotarev as zo

M0 = 1.4


@functools.lru_cache(maxsize=None)
def lib():
    from paper_1501_01855_gb300 import build, binding
    build.build()
    binding.load()
    return binding


@functools.lru_cache(maxsize=4)
def dense_4444(seed=1001):
    """Dense K, its exact sign and spectrum on the 4^4 config-1 lattice (oracle)."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_links(dims, 0.3, seed)
    Kd = wilson.dense_K(U, M0)
    S, w = overlap.dense_sign(Kd)
    return U, Kd, S, w


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def ctx(dims, links, mu=0.05, n_poles=16, eps=1e-10, a=None, b=None, **kw):
    B = lib()
    p = B.ovl_params_default()
    if a is not None:
        p.a_override = a
    if b is not None:
        p.b_override = b
    for k, v in kw.items():
        setattr(p, k, v)
    return B.Overlap(dims, links, M0, mu, n_poles, eps, params=p)
