"""Seeded synthetic inputs shared by the tests and bench.py.

Holds none of the method's arithmetic: random perturbations, probe points,
directions and instance sizes only (numpy default_rng, fixed seeds).  Both the
oracle checks and the CUDA parity tests draw their inputs from here.
"""
import numpy as np


def perturbation(shape, seed, scale):
    """Uniform noise in [-scale, scale] of the given shape (float64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=shape)


def smooth_perturbation(shape, seed, scale):
    """Per-variable random amplitudes for a smooth nodal bump (values only; the
    caller multiplies them onto its own nodal field)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=shape)


def probes(count, seed, lo=0.0, hi=1000.0):
    """Probe points uniform in [lo, hi]^2."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(count, 2))


def directions(count, dim, seed):
    """Unit-norm Gaussian directions."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((count, dim))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def instance_sizes(count, seed, lo=9, hi=81):
    """Integer grid sides uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count)


def uniform_values(count, seed, lo, hi):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=count)


def normal_values(count, seed, scale):
    """Gaussian values N(0, scale^2)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, size=count)
