"""The algorithm of the GPU spline sweep, restated in numpy and checked on
the CPU against the oracle's cyclic solve: the symbol of the cyclic system
factors as (S^-1 + 4 + S)/6 = (1 + zS)(1 + zS^-1)/(6z), z = 2 - sqrt(3), so
the coefficients are 6z times two periodic first-order recurrences; each of
four chunks of a line starts its recurrence W points early from zero
(W = 32 in FP64, 16 in FP32).  The truncation must stay below the rounding
of the working precision for every line length, including lines shorter
than W (the warm-up wraps several times)."""
import numpy as np
import pytest

from inputs import rng


def _chunked_coeffs(u, W, dtype):
    n = u.size
    z = dtype(2.0 - np.sqrt(3.0))
    u = u.astype(dtype)
    C = -(-n // 4)
    y = np.zeros(n, dtype)
    for c in range(4):
        ib, ie = min(c * C, n), min(c * C + C, n)
        if ib >= ie:
            continue
        acc, k = dtype(0), (ib - W) % n
        for _ in range(W):
            acc = u[k] - z * acc
            k = (k + 1) % n
        for i in range(ib, ie):
            acc = u[i] - z * acc
            y[i] = acc
    w = np.zeros(n, dtype)
    for c in range(4):
        ib, ie = min(c * C, n), min(c * C + C, n)
        if ib >= ie:
            continue
        acc, k = dtype(0), (ie - 1 + W) % n
        for _ in range(W):
            acc = y[k] - z * acc
            k = (k - 1) % n
        for i in range(ie - 1, ib - 1, -1):
            acc = y[i] - z * acc
            w[i] = dtype(6) * z * acc
    return w


@pytest.mark.parametrize("n", [3, 4, 5, 8, 31, 37, 128, 300])
def test_chunked_recurrences_match_the_cyclic_solve(orc, n):
    u = rng(40 + n).standard_normal(n)
    ref = orc.spline_coeffs(u)
    w64 = _chunked_coeffs(u, 32, np.float64)
    assert np.abs(w64 - ref).max() < 1e-14 * np.abs(ref).max()
    w32 = _chunked_coeffs(u, 16, np.float32)
    assert np.abs(w32.astype(np.float64) - ref).max() < 2e-6 * np.abs(ref).max()


def test_truncation_bound():
    z = 2.0 - np.sqrt(3.0)
    assert z ** 33 / (1 - z) < 2.0 ** -61
    assert z ** 17 / (1 - z) < 2.0 ** -31
