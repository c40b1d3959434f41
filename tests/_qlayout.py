"""Layout conversions used by the tests only.

The library stores a quaternion tensor as (2, rows, cols, p, 2) "complex-pair
planes" (plane 0 = a + b i, plane 1 = c + d i; last axis real/imag).  The
oracle works on (4, rows, cols, p) real components (a, b, c, d).
"""
import numpy as np


def planes_to_comp(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return np.stack([x[0, ..., 0], x[0, ..., 1], x[1, ..., 0], x[1, ..., 1]])


def comp_to_planes(q, dtype=np.float32) -> np.ndarray:
    q = np.asarray(q)
    out = np.empty((2,) + q.shape[1:] + (2,), dtype=dtype)
    out[0, ..., 0], out[0, ..., 1], out[1, ..., 0], out[1, ..., 1] = q[0], q[1], q[2], q[3]
    return out
