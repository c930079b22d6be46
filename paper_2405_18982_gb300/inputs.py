"""Seeded synthetic inputs shared by the tests, the oracle runs and the
benchmark.  Only random numbers live here (NumPy PCG64 in FP64): no
arithmetic of the discretisation or the solver, so both the CUDA path and
the oracle receive identical bits from a source independent of either.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def uniform(seed, n, lo=-1.0, hi=1.0):
    """n values U[lo, hi) (FP64)."""
    return rng(seed).uniform(lo, hi, size=n)


def normal(seed, n):
    """n values N(0, 1) (FP64)."""
    return rng(seed).standard_normal(n)


def normal_columns(seeds, n):
    """One N(0,1) column per seed, stacked (len(seeds), n)."""
    return np.stack([normal(s, n) for s in seeds])


def ragged_problems(seed, count=64, levels=(5, 9), degrees=(2, 6)):
    """(log2_cells, degree) pairs of a ragged batch of independent 2D problems:
    log2_cells uniform in levels, degree uniform in degrees (inclusive)."""
    g = rng(seed)
    L = g.integers(levels[0], levels[1] + 1, size=count)
    k = g.integers(degrees[0], degrees[1] + 1, size=count)
    return [(int(a), int(b)) for a, b in zip(L, k)]


def scalar_uniform(seed, lo, hi):
    return float(rng(seed).uniform(lo, hi))
