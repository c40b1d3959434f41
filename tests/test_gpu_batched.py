"""Batched products (qtp_forward_batched) through the C ABI against the oracle."""
import numpy as np
import pytest

import oracle as Q
from paper_2212_14318_gb300 import synth
from tests._gpu import assert_close, rel_fro, to_dev, to_host
from tests._qlayout import planes_to_comp

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
ELEM_TOL = 1e-4

# mixed shapes: specialised and generic tube lengths, ragged tiles, tiny and wide products
MIXED = [(8, 8, 8, 16), (17, 9, 13, 3), (33, 65, 31, 7), (130, 40, 150, 8), (5, 3, 4, 2), (1, 1, 1, 1),
         (20, 30, 40, 12), (16, 16, 16, 31), (40, 24, 36, 64), (13, 7, 11, 100), (64, 48, 80, 128),
         (9, 11, 10, 97), (3, 5, 7, 1), (70, 1, 70, 5), (24, 20, 28, 32), (12, 12, 12, 8),
         # s well above m: computed as C^T = B^T A^T on the tensor cores (several
         # row tiles over s; two column tiles over m in the second)
         (20, 30, 200, 8), (150, 40, 300, 4), (5, 17, 260, 12)]


def _check_all(shapes, As, Bs, Cs, what):
    for i, (m, n, s, p) in enumerate(shapes):
        Aq, Bq = planes_to_comp(As[i]), planes_to_comp(Bs[i])
        if p <= 32:
            ref = Q.tprod_def(Aq, Bq)
            assert_close(to_host(Cs[i]), ref, REL_TOL, ELEM_TOL, f"{what} product {i} {m}x{n}x{s}x{p}")
        else:
            cols = synth.sample_columns(s, 4)
            assert_close(to_host(Cs[i])[:, :, cols], Q.tprod_def_columns(Aq, Bq, cols), REL_TOL, ELEM_TOL,
                         f"{what} product {i} {m}x{n}x{s}x{p}")


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
@pytest.mark.parametrize("graph", [True, False])
def test_mixed_batch_matches_oracle(precision, graph):
    import torch
    from paper_2212_14318_gb300 import qtp
    As = [synth.quat_normal(m, n, p, 900 + i) for i, (m, n, s, p) in enumerate(MIXED)]
    Bs = [synth.quat_normal(n, s, p, 1900 + i) for i, (m, n, s, p) in enumerate(MIXED)]
    dA, dB = [to_dev(a) for a in As], [to_dev(b) for b in Bs]
    plan = qtp.BatchPlan(MIXED, precision, graph=graph)
    Cs = plan.forward(dA, dB)
    plan.sync()
    _check_all(MIXED, As, Bs, Cs, f"{precision} graph={graph}")
    # replay with other inputs and outputs (new pointers, same workspace), then with a new workspace
    As2 = [a[::-1].copy() for a in As]                  # swap the Cayley-Dickson planes
    dA2 = [to_dev(a) for a in As2]
    Cs2 = plan.forward(dA2, dB)
    plan.sync()
    _check_all(MIXED, As2, Bs, Cs2, f"{precision} replay")
    ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device="cuda")
    Cs3 = plan.forward(dA, dB, workspace=ws)
    plan.sync()
    for c1, c3 in zip(Cs, Cs3):
        np.testing.assert_array_equal(to_host(c1), to_host(c3))


def test_batch_matches_single_product_entry_point():
    """Same split-BF16 arithmetic through both entry points (the single-product
    path's one-CTA FP32 route for tiny products is switched off here)."""
    import os
    from paper_2212_14318_gb300 import qtp
    shapes = MIXED[:6]
    As = [to_dev(synth.quat_normal(m, n, p, 50 + i)) for i, (m, n, s, p) in enumerate(shapes)]
    Bs = [to_dev(synth.quat_normal(n, s, p, 60 + i)) for i, (m, n, s, p) in enumerate(shapes)]
    Cs = qtp.BatchPlan(shapes, "bf16x3").forward(As, Bs)
    os.environ["QTP_NO_FUSED"] = "1"
    try:
        for i, (m, n, s, p) in enumerate(shapes):
            ref = qtp.Plan(m, n, s, p, "bf16x3").forward(As[i], Bs[i])
            assert rel_fro(to_host(Cs[i]), to_host(ref)) <= 1e-6
    finally:
        del os.environ["QTP_NO_FUSED"]


def test_batch_workload_4096_products_each_checked():
    """4096 products, m, n, s log-uniform in [16, 256], p in {8,12,16,31,32,64,100,128};
    one persistent launch per stage replayed from a CUDA graph; every product is
    checked against the oracle on two sampled entries."""
    import torch
    from paper_2212_14318_gb300 import qtp
    shapes = synth.batch_shapes()
    As, Bs = synth.batch_tensors(shapes)
    plan = qtp.BatchPlan(shapes, "bf16x3")
    Cs = plan.forward(As, Bs)
    plan.sync()
    rng = np.random.default_rng(synth.SEED_SAMPLE)
    num, den = 0.0, 0.0
    worst = 0.0
    for i, (m, n, s, p) in enumerate(shapes):
        ii, tt, kk = rng.integers(0, m, 2), rng.integers(0, s, 2), rng.integers(0, p, 2)
        arow = As[i][:, ii].cpu().numpy()                       # (2, 2, n, p, 2)
        bcol = Bs[i][:, :, tt].cpu().numpy()                    # (2, n, 2, p, 2)
        got = Cs[i][:, ii, tt, kk].cpu().numpy().astype(np.float64)   # (2, 2, 2)
        for e in range(2):
            a = planes_to_comp(arow[:, e:e + 1])                # (4, 1, n, p)
            b = planes_to_comp(bcol[:, :, e:e + 1])             # (4, n, 1, p)
            ref = Q.tprod_def_entries(a, b, [0], [0], [kk[e]])[:, 0]
            g = np.array([got[0, e, 0], got[0, e, 1], got[1, e, 0], got[1, e, 1]])
            err = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
            worst = max(worst, err)
            num += np.sum((g - ref) ** 2)
            den += np.sum(ref ** 2)
    assert np.sqrt(num / den) <= REL_TOL, np.sqrt(num / den)
    assert worst <= 1e-4, worst
    del As, Bs, Cs
    torch.cuda.empty_cache()


@pytest.mark.parametrize("graph", [True, False])
def test_batch_stage_tracing(graph):
    from paper_2212_14318_gb300 import qtp
    shapes = MIXED[:4]
    As = [to_dev(synth.quat_normal(m, n, p, 70 + i)) for i, (m, n, s, p) in enumerate(shapes)]
    Bs = [to_dev(synth.quat_normal(n, s, p, 80 + i)) for i, (m, n, s, p) in enumerate(shapes)]
    plan = qtp.BatchPlan(shapes, "bf16x3", graph=graph)
    plan.set_tracing(True)
    plan.forward(As, Bs)
    t = plan.stage_times()
    assert len(t) == 3 and all(x > 0 for x in t)
    plan.set_tracing(False)
    plan.forward(As, Bs)
    plan.sync()


def test_bound_batch_repeats_with_new_contents():
    """BatchPlan.bind validates the tensors once; each bound forward() is one
    qtp_forward_batched call on the same pointers.  New input contents
    written in place give the new products (oracle), and the bound result
    equals the unbound call's bit for bit."""
    from paper_2212_14318_gb300 import qtp
    shapes = MIXED[:8]
    As = [synth.quat_normal(m, n, p, 700 + i) for i, (m, n, s, p) in enumerate(shapes)]
    Bs = [synth.quat_normal(n, s, p, 800 + i) for i, (m, n, s, p) in enumerate(shapes)]
    dA, dB = [to_dev(a) for a in As], [to_dev(b) for b in Bs]
    plan = qtp.BatchPlan(shapes, "bf16x3")
    bound = plan.bind(dA, dB)
    Cs = bound.forward()
    plan.sync()
    _check_all(shapes, As, Bs, Cs, "bound")
    ref = plan.forward(dA, dB)
    plan.sync()
    for c, r in zip(Cs, ref):
        np.testing.assert_array_equal(to_host(c), to_host(r))
    As2 = [-a for a in As]
    for t, a in zip(dA, As2):
        t.copy_(to_dev(a))
    bound.forward()
    plan.sync()
    _check_all(shapes, As2, Bs, bound.Cs, "bound, new contents")


# products of the batch routing tests: narrow, wide (min(m, s) >= 64 / 128),
# transposed, and one with a long reduction
ROUTE_SHAPES = [(8, 8, 8, 16), (150, 40, 300, 4), (70, 33, 90, 12), (130, 64, 140, 8), (20, 30, 200, 8),
                (64, 500, 72, 4), (16, 16, 16, 31), (96, 48, 96, 32)]


@pytest.mark.parametrize("route_min", ["0", "64", "128"])
def test_routed_products_match_oracle(route_min, monkeypatch):
    """Products routed to the single-product kernel (all of them at 0; those
    with min(m, s) >= 64 or 128), launched over the plan's auxiliary streams
    inside the graph, against the oracle; a second replay repeats them."""
    from paper_2212_14318_gb300 import qtp
    monkeypatch.setenv("QTP_BATCH_ROUTE_MIN", route_min)
    As = [synth.quat_normal(m, n, p, 610 + i) for i, (m, n, s, p) in enumerate(ROUTE_SHAPES)]
    Bs = [synth.quat_normal(n, s, p, 620 + i) for i, (m, n, s, p) in enumerate(ROUTE_SHAPES)]
    plan = qtp.BatchPlan(ROUTE_SHAPES, "bf16x3")
    assert plan.route()[0] == int(route_min)
    dA, dB = [to_dev(a) for a in As], [to_dev(b) for b in Bs]
    Cs = plan.forward(dA, dB)
    plan.sync()
    _check_all(ROUTE_SHAPES, As, Bs, Cs, f"route_min={route_min}")
    first = [to_host(c) for c in Cs]
    plan.forward(dA, dB, Cs)
    plan.sync()
    for c, f in zip(Cs, first):
        np.testing.assert_array_equal(to_host(c), f)


def test_autotuned_batch_routing():
    """QTP_BATCH_AUTOTUNE times the products for each candidate threshold and
    keeps the fastest; the tuned plan matches the oracle and a second plan of
    the same shapes reuses the choice."""
    from paper_2212_14318_gb300 import qtp
    shapes = ROUTE_SHAPES * 3
    As = [synth.quat_normal(m, n, p, 630 + i) for i, (m, n, s, p) in enumerate(shapes)]
    Bs = [synth.quat_normal(n, s, p, 660 + i) for i, (m, n, s, p) in enumerate(shapes)]
    plan = qtp.BatchPlan(shapes, "bf16x3", autotune=True)
    route_min, times = plan.route()
    assert len(times) == 6 and all(t > 0 for t in times), times
    assert route_min in (2**31 - 1, 192, 128, 96, 64, 48)
    assert times[[2**31 - 1, 192, 128, 96, 64, 48].index(route_min)] == min(times)
    Cs = plan.forward([to_dev(a) for a in As], [to_dev(b) for b in Bs])
    plan.sync()
    _check_all(shapes, As, Bs, Cs, "autotuned routing")
    assert qtp.BatchPlan(shapes, "bf16x3", autotune=True).route()[0] == route_min
