"""Seeded synthetic inputs for the quaternion T-product workloads.

This module holds random-number generation and shapes only: none of the
T-product's arithmetic.  Both the CUDA path's tests/bench and the FP64 oracle
draw their inputs from here.  It imports nothing else from the package.

Every tensor is returned in the library's layout, "tube-contiguous
complex-pair planes": a float32/float64 array of shape (2, rows, cols, p, 2)
where plane 0 holds X1 = a + b i and plane 1 holds X2 = c + d i of the
quaternion a + b i + c j + d k, and the last axis is (real, imag).

Workloads (the paper uses random tensors, Sec. 5 Example 5.1; its colour-video
motivation, Sec. 1, is mirrored by a pixel-like pure-quaternion A):

* small      A 8x8x16,  B 8x8x16, N(0,1) components
* video      A 240x320x64 pure quaternion (a = 0, b, c, d ~ U[0, 1]),
             B 320x240x64 N(0,1)
* precision  A 1024x1024x128, B 1024x1024x128, N(0,1)
* batch      4096 problems, m, n, s = round(exp(U(ln 16, ln 256))),
             p uniform over {8, 12, 16, 31, 32, 64, 100, 128}
* diff       A 128x64x32, B 64x128x32, target T 128x128x32, N(0,1)
* long1000, long1024, long4096  A, B 64x64xp N(0,1): long tubes (long
             videos), the two-pass transforms

Seeds: 0 for A, 1 for B, 2 for T, 3 for sampled output positions, 4 for the
batch shape draw.
"""
from __future__ import annotations

import numpy as np

SEED_A, SEED_B, SEED_T, SEED_SAMPLE, SEED_BATCH = 0, 1, 2, 3, 4

WORKLOADS = {
    "small": dict(m=8, n=8, s=8, p=16, a_kind="normal"),
    "video": dict(m=240, n=320, s=240, p=64, a_kind="pixel"),
    "precision": dict(m=1024, n=1024, s=1024, p=128, a_kind="normal"),
    "diff": dict(m=128, n=64, s=128, p=32, a_kind="normal"),
    "long1000": dict(m=64, n=64, s=64, p=1000, a_kind="normal"),
    "long1024": dict(m=64, n=64, s=64, p=1024, a_kind="normal"),
    "long4096": dict(m=64, n=64, s=64, p=4096, a_kind="normal"),
}

BATCH_P_CHOICES = (8, 12, 16, 31, 32, 64, 100, 128)


def quat_normal(rows: int, cols: int, p: int, seed: int, dtype=np.float32) -> np.ndarray:
    """i.i.d. N(0,1) quaternion tensor in plane layout (2, rows, cols, p, 2)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((2, rows, cols, p, 2), dtype=np.dtype(dtype).type)


def quat_pixel(rows: int, cols: int, p: int, seed: int, dtype=np.float32) -> np.ndarray:
    """Pure quaternion b i + c j + d k with b, c, d ~ U[0, 1] (colour pixels).

    Plane 0 = (a, b) = (0, b); plane 1 = (c, d).
    """
    rng = np.random.default_rng(seed)
    x = rng.random((2, rows, cols, p, 2), dtype=np.dtype(dtype).type)
    x[0, ..., 0] = 0.0
    return x


def workload(name: str, dtype=np.float32):
    """(A, B) for a named single-product workload, in plane layout."""
    w = WORKLOADS[name]
    m, n, s, p = w["m"], w["n"], w["s"], w["p"]
    if w["a_kind"] == "pixel":
        A = quat_pixel(m, n, p, SEED_A, dtype)
    else:
        A = quat_normal(m, n, p, SEED_A, dtype)
    B = quat_normal(n, s, p, SEED_B, dtype)
    return A, B


def target(name: str, dtype=np.float32) -> np.ndarray:
    """Target tensor T (m x s x p) for the loss ||A*B - T||^2."""
    w = WORKLOADS[name]
    return quat_normal(w["m"], w["s"], w["p"], SEED_T, dtype)


def batch_shapes(count: int = 4096, seed: int = SEED_BATCH, lo: int = 16, hi: int = 256,
                 p_choices=BATCH_P_CHOICES):
    """Shapes (m, n, s, p) for the batched workload, log-uniform m, n, s."""
    rng = np.random.default_rng(seed)
    mns = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=(count, 3)))).astype(np.int64)
    ps = rng.choice(np.asarray(p_choices, dtype=np.int64), size=count)
    return [(int(a), int(b), int(c), int(d)) for (a, b, c), d in zip(mns, ps)]


def sample_positions(m: int, s: int, p: int, count: int, seed: int = SEED_SAMPLE):
    """Random output positions (i, t, k) for sampled checks of C."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, m, count), rng.integers(0, s, count), rng.integers(0, p, count))


def sample_columns(s: int, count: int, seed: int = SEED_SAMPLE):
    """Distinct random lateral column indices t for sampled checks of C(:, t, :)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(s, size=min(count, s), replace=False))


def batch_tensors(shapes, seed: int = SEED_A, device="cuda"):
    """N(0,1) inputs (A_i, B_i) for a batch, drawn on the device by torch's
    seeded generator (the batch holds tens of GB); plane layout per tensor."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    As, Bs = [], []
    for (m, n, s, p) in shapes:
        As.append(torch.randn((2, m, n, p, 2), generator=g, device=device, dtype=torch.float32))
        Bs.append(torch.randn((2, n, s, p, 2), generator=g, device=device, dtype=torch.float32))
    return As, Bs
