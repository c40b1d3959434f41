"""Split-BF16 accuracy for long reductions (Thm 5.1 Step 2, through the C ABI).

The per-frequency products reduce over K = n (forward), s (dA) or m (dB) per
half of the m x 2n x 2s complex product.  The tensor core accumulates in FP32
with an error that grows with the number of MMAs folded into one TMEM
accumulator, so the kernel switches accumulator mode with K: one pair up to
384, split (hi.hi apart from the corrections) up to 1024, and promotion of the
partial sums to an FP32 running sum every 32 K steps beyond.  Every case here
is compared element by element with the FP64 oracle's definition
(Definition 2.3) at the same bound as every other parity test: relative
Frobenius error <= 1e-5 and every |x - ref| <= 1e-4 * rms(ref).
"""
import numpy as np
import pytest

import oracle as Q
from paper_2212_14318_gb300 import synth
from tests._gpu import assert_close, to_dev, to_host
from tests._qlayout import planes_to_comp

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
ELEM_TOL = 1e-4

# (m, n, s, p): split accumulators (K = 1000), promoted accumulators with a
# ragged last segment (1500 = 93.75 K steps of 16 per half), K = 4096 and
# K = 16384 (32 promotions per tile)
FORWARD = [(24, 1000, 20, 3), (20, 1500, 24, 2), (48, 4096, 40, 4), (16, 16384, 16, 2)]


def _qtp():
    import torch
    from paper_2212_14318_gb300 import qtp
    assert torch.cuda.is_available()
    return qtp


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
@pytest.mark.parametrize("m,n,s,p", FORWARD)
def test_forward_long_reduction(precision, m, n, s, p):
    qtp = _qtp()
    A = synth.quat_normal(m, n, p, seed=n + 1)
    B = synth.quat_normal(n, s, p, seed=n + 2)
    plan = qtp.Plan(m, n, s, p, precision)
    C = to_host(plan.forward(to_dev(A), to_dev(B)))
    plan.sync()
    ref = Q.tprod_def(planes_to_comp(A), planes_to_comp(B))
    rf = assert_close(C, ref, REL_TOL, ELEM_TOL, f"{precision} forward K={n}")
    print(f"forward {precision} {m}x{n}x{s}x{p}: rel err {rf:.2e}, tiles {plan.tiles()}")


@pytest.mark.parametrize("m,n,s,p", [(40, 24, 4096, 4), (4096, 24, 40, 4), (36, 20, 1300, 3)])
def test_backward_long_reduction(m, n, s, p):
    """dA reduces over s, dB over m: one long reduction per kind."""
    qtp = _qtp()
    A = synth.quat_normal(m, n, p, seed=3 * s + 1)
    B = synth.quat_normal(n, s, p, seed=3 * s + 2)
    G = synth.quat_normal(m, s, p, seed=3 * s + 3)
    plan = qtp.Plan(m, n, s, p, "bf16x3")
    dA, dB = plan.backward(to_dev(G), to_dev(A), to_dev(B))
    plan.sync()
    Aq, Bq, Gq = planes_to_comp(A), planes_to_comp(B), planes_to_comp(G)
    ea = assert_close(to_host(dA), Q.tprod_def(Gq, Q.conj_transpose(Bq)), REL_TOL, ELEM_TOL, f"dA K={s}")
    eb = assert_close(to_host(dB), Q.tprod_def(Q.conj_transpose(Aq), Gq), REL_TOL, ELEM_TOL, f"dB K={m}")
    print(f"backward {m}x{n}x{s}x{p}: dA rel err {ea:.2e}, dB rel err {eb:.2e}")


def test_autotuned_long_reduction():
    """An autotuned plan at K = 4096 may only choose promoted accumulators for
    the forward (the other modes exceed 1e-5 there), and stays within 1e-5."""
    qtp = _qtp()
    m, n, s, p = 48, 4096, 40, 4
    A = synth.quat_normal(m, n, p, seed=41)
    B = synth.quat_normal(n, s, p, seed=42)
    plan = qtp.Plan(m, n, s, p, "bf16x3", autotune=True)
    tiles = plan.tiles()
    assert tiles[0] == 4, tiles  # 128 wide, promoted accumulators
    C = to_host(plan.forward(to_dev(A), to_dev(B)))
    plan.sync()
    assert_close(C, Q.tprod_def(planes_to_comp(A), planes_to_comp(B)), REL_TOL, ELEM_TOL, "autotuned K=4096")


def test_batched_long_reduction():
    """A batch whose products with n > 384 leave the grouped kernel for the
    single-product kernel (split at n = 600, promoted at n = 1100), mixed
    with products the grouped kernel keeps; graph replay twice."""
    qtp = _qtp()
    shapes = [(20, 600, 30, 8), (16, 16, 16, 8), (24, 1100, 20, 4), (40, 30, 50, 12), (8, 2000, 8, 3)]
    As = [synth.quat_normal(a, b, q, 300 + i) for i, (a, b, c, q) in enumerate(shapes)]
    Bs = [synth.quat_normal(b, c, q, 400 + i) for i, (a, b, c, q) in enumerate(shapes)]
    plan = qtp.BatchPlan(shapes, "bf16x3")
    dA, dB = [to_dev(a) for a in As], [to_dev(b) for b in Bs]
    Cs = plan.forward(dA, dB)
    plan.sync()
    first = [to_host(c) for c in Cs]
    plan.forward(dA, dB, Cs)
    plan.sync()
    for i, (a, b, c, q) in enumerate(shapes):
        np.testing.assert_array_equal(to_host(Cs[i]), first[i])
        ref = Q.tprod_def(planes_to_comp(As[i]), planes_to_comp(Bs[i]))
        assert_close(first[i], ref, REL_TOL, ELEM_TOL, f"batched product {i} {shapes[i]}")
