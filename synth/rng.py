"""Seeded random generators for synthetic inputs (numpy PCG64).

Nothing here computes any step of the method: it only draws numbers that are
then passed to both the oracle and the CUDA library as inputs.
"""
import numpy as np


def seeded_uniform(seed, shape, lo=0.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def seeded_normal(seed, shape, scale=1.0):
    return np.random.default_rng(seed).normal(0.0, scale, size=shape)


def mlp_init(seed, k_in, hidden=64):
    """He-uniform initial weights of the K -> 64 -> 64 -> 1 indicator network.

    Returns a dict of float64 arrays: W1 (hidden, K), b1 (hidden), W2 (hidden, hidden),
    b2 (hidden), W3 (1, hidden), b3 (1).
    """
    rng = np.random.default_rng(seed)

    def he(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=shape)

    return {
        'W1': he(k_in, (hidden, k_in)), 'b1': np.zeros(hidden),
        'W2': he(hidden, (hidden, hidden)), 'b2': np.zeros(hidden),
        'W3': he(hidden, (1, hidden)) * 0.5, 'b3': np.zeros(1),
    }
