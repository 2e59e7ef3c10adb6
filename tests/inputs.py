"""Seeded synthetic inputs shared by the oracle side and the CUDA side of the parity tests.

Holds no arithmetic of the method: only random numbers with a fixed seed.
"""
import numpy as np


def random_amplitudes(n, seed=1234, scale=0.05):
    """n amplitudes drawn from N(0, scale^2) (converged amplitudes are of order 1e-2)."""
    return np.random.default_rng(seed).normal(0.0, scale, n)
