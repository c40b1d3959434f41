"""Autotuned tile choice (QTP_PLAN_AUTOTUNE): valid, accurate, cached."""
import os

import pytest

import oracle as Q
from paper_2212_14318_gb300 import synth
from tests._gpu import assert_close, to_dev, to_host
from tests._qlayout import planes_to_comp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,s,p", [(200, 96, 200, 8), (40, 500, 60, 4)])
def test_autotuned_plan_is_accurate_and_respects_the_accuracy_rule(m, n, s, p, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("QTP_AUTOTUNE_CACHE", str(cache))
    from paper_2212_14318_gb300 import qtp
    A = synth.quat_normal(m, n, p, 3)
    B = synth.quat_normal(n, s, p, 4)
    plan = qtp.Plan(m, n, s, p, "bf16x3", autotune=True)
    tiles = plan.tiles()
    assert all(t in (1, 2, 3, 4) for t in tiles), tiles
    # the accuracy rule for the forward product's reduction K = n: one
    # accumulator pair (tiles 1, 2) only up to 384, split accumulators (3) up to
    # 1024, promoted ones (4) at any length
    if n > 384:
        assert tiles[0] in (3, 4), tiles
    if n > 1024:
        assert tiles[0] == 4, tiles
    C = to_host(plan.forward(to_dev(A), to_dev(B)))
    plan.sync()
    assert_close(C, Q.tprod_def(planes_to_comp(A), planes_to_comp(B)), 1e-5, 1e-4, "autotuned")
    G = synth.quat_normal(m, s, p, 5)
    dA, dB = plan.backward(to_dev(G), to_dev(A), to_dev(B))
    Aq, Bq, Gq = planes_to_comp(A), planes_to_comp(B), planes_to_comp(G)
    assert_close(to_host(dA), Q.tprod_def(Gq, Q.conj_transpose(Bq)), 1e-5, 1e-4, "autotuned dA")
    assert_close(to_host(dB), Q.tprod_def(Q.conj_transpose(Aq), Gq), 1e-5, 1e-4, "autotuned dB")
    # a second plan of the same shape reuses the choice
    assert qtp.Plan(m, n, s, p, "bf16x3", autotune=True).tiles() == tiles
    if os.path.exists(cache):
        lines = cache.read_text().split("\n")
        assert any(f":{m}:{n}:{s}:{p}:1 " in ln for ln in lines)


@pytest.mark.parametrize("m,n,s,p", [(6, 5, 7, 1024), (4, 6, 5, 1000)])
def test_autotuned_transform_forms(m, n, s, p, tmp_path, monkeypatch):
    """With p > 128 the autotuner also times the tube transform forms (one
    kernel, runtime two-pass, compile-time two-pass) per direction; the plan
    with its choice matches the oracle's FP64 Algorithm 5.1, forward and
    backward."""
    monkeypatch.setenv("QTP_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    from paper_2212_14318_gb300 import qtp
    A = synth.quat_normal(m, n, p, 13)
    B = synth.quat_normal(n, s, p, 14)
    G = synth.quat_normal(m, s, p, 15)
    for precision in ("bf16x3", "fp32"):
        plan = qtp.Plan(m, n, s, p, precision, autotune=True)
        fwd, bwd = plan.launch_count()
        # transforms in one or two launches each; the split-BF16 forward of these
        # small products adds the grouped-tile products' record copy
        extra = 1 if precision == "bf16x3" else 0
        assert fwd - extra in (3, 4, 5) and bwd in (5, 6, 7, 8), (fwd, bwd)
        C = to_host(plan.forward(to_dev(A), to_dev(B)))
        plan.sync()
        Aq, Bq, Gq = planes_to_comp(A), planes_to_comp(B), planes_to_comp(G)
        assert_close(C, Q.alg51(Aq, Bq), 1e-5, 1e-4, f"autotuned forms {precision} p={p}")
        dA, dB = plan.backward(to_dev(G), to_dev(A), to_dev(B))
        plan.sync()
        assert_close(to_host(dA), Q.alg51(Gq, Q.conj_transpose(Bq)), 1e-5, 1e-4, f"autotuned forms dA {precision}")
        assert_close(to_host(dB), Q.alg51(Q.conj_transpose(Aq), Gq), 1e-5, 1e-4, f"autotuned forms dB {precision}")
