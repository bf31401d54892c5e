"""Seeded synthetic inputs shared by the oracle and CUDA parity tests.

This module only draws random numbers and builds grid descriptions; it holds
none of the method's arithmetic.
"""
import numpy as np

# Domains of the paper's workloads (Sec. 4 nonlinear Landau, Sec. 5 two-stream)
LANDAU_LO = (0.0, 0.0, -6.0, -6.0)
LANDAU_HI = (4 * np.pi, 4 * np.pi, 6.0, 6.0)
TSI_LO = (0.0, 0.0, -9.0, -9.0)
TSI_HI = (10 * np.pi, 10 * np.pi, 9.0, 9.0)


def rng(seed):
    return np.random.default_rng(seed)


def random_f(shape, seed, positive=False):
    r = rng(seed)
    a = r.standard_normal(shape)
    if positive:
        a = np.abs(a) + 0.1
    return np.ascontiguousarray(a, dtype=np.float64)


def random_field(shape, seed, scale=1.0):
    r = rng(seed)
    return np.ascontiguousarray(scale * r.standard_normal(shape), dtype=np.float64)


def smooth_field(shape, seed, scale=1.0):
    """Smooth periodic field on a (D2, D1) node grid: a few random Fourier modes."""
    r = rng(seed)
    D2, D1 = shape
    y, x = np.meshgrid(np.linspace(0, 2 * np.pi, D2, endpoint=False),
                       np.linspace(0, 2 * np.pi, D1, endpoint=False), indexing="ij")
    out = np.zeros(shape)
    for _ in range(4):
        m1, m2 = r.integers(-2, 3, size=2)
        out += r.standard_normal() * np.cos(m1 * x + m2 * y + r.uniform(0, 2 * np.pi))
    return np.ascontiguousarray(scale * out)
