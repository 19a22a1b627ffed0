"""Small shared fixtures for the oracle pin tests (test infrastructure)."""
import functools

import numpy as np

import synth
from oracle import wilson, overlap


@functools.lru_cache(maxsize=8)
def dense_setup(dims, eps=0.3, seed=1001, m0=1.4, antiperiodic_t=False):
    U = synth.gauge_links(dims, eps, seed)
    Kd = wilson.dense_K(U, m0, antiperiodic_t)
    S, w = overlap.dense_sign(Kd)
    return U, Kd, S, w
