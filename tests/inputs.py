"""Seeded synthetic inputs shared by the oracle side and the CUDA side of the parity tests.

Holds no arithmetic of the method: only random numbers with a fixed seed.
"""
import numpy as np


def random_amplitudes(n, seed=1234, scale=0.05):
    """n amplitudes drawn from N(0, scale^2) (converged amplitudes are of order 1e-2)."""
    return np.random.default_rng(seed).normal(0.0, scale, n)


def random_mlp(n=64, seed=0, nparam=None):
    """A parameter blob for the warm-start network (layout of oracle.mlp / pnm_mlp_*), with
    weights ~ N(0, 1/fan_in), small biases, unit feature normalisation; plus n random
    feature rows (32 columns, the last 10 zero as in real features) and targets."""
    F, H = 32, 128
    rng = np.random.default_rng(seed)
    parts = [np.zeros(F), np.ones(F), np.ones(1), np.zeros(3),
             rng.normal(0, 1 / np.sqrt(F), (H, F)).ravel(), rng.normal(0, 0.1, H),
             rng.normal(0, 1 / np.sqrt(H), (H, H)).ravel(), rng.normal(0, 0.1, H),
             rng.normal(0, 1 / np.sqrt(H), (H, H)).ravel(), rng.normal(0, 0.1, H),
             rng.normal(0, 1 / np.sqrt(H), H), rng.normal(0, 0.1, 1)]
    blob = np.concatenate(parts).astype(np.float32)
    if nparam is not None:
        assert blob.size == nparam
    X = rng.normal(0, 1, (n, F)).astype(np.float32)
    X[:, 22:] = 0
    T = rng.normal(0, 1, n).astype(np.float32)
    return blob, X, T
