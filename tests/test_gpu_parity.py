"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every case feeds the same seeded FP32 inputs to libqtp and (cast to FP64) to
the oracle's definition-based T-product, then compares element by element.
Tolerance: relative Frobenius error <= 1e-5 (FP32 outputs) and every element
within 1e-4 * rms of the reference.
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
PRECISIONS = ["fp32", "bf16x3"]

# (m, n, s, p): edge sizes, ragged tails over several tiles, every radix path
SHAPES = [
    (1, 1, 1, 1), (3, 5, 7, 1), (5, 3, 4, 2), (17, 9, 13, 3), (8, 8, 8, 16), (20, 30, 40, 12),
    (16, 16, 16, 31), (33, 65, 31, 7), (1, 70, 1, 8), (70, 1, 70, 5), (130, 40, 260, 8),
    (40, 24, 36, 64), (13, 7, 11, 100), (64, 48, 80, 128), (9, 11, 10, 97), (150, 70, 300, 16),
    (20, 12, 24, 32), (24, 500, 40, 4),   # K = 500: split accumulators
]


def _qtp():
    import torch
    from paper_2212_14318_gb300 import qtp
    assert torch.cuda.is_available()
    return qtp


def _inputs(m, n, s, p, seed):
    A = synth.quat_normal(m, n, p, seed)
    B = synth.quat_normal(n, s, p, seed + 1000)
    return A, B


def _oracle(A, B, cols=None):
    Aq, Bq = planes_to_comp(A), planes_to_comp(B)
    if cols is None:
        return Q.tprod_def(Aq, Bq)
    return Q.tprod_def_columns(Aq, Bq, cols)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("m,n,s,p", SHAPES)
def test_forward_matches_oracle(precision, m, n, s, p):
    qtp = _qtp()
    A, B = _inputs(m, n, s, p, seed=m * 7 + n * 3 + p)
    plan = qtp.Plan(m, n, s, p, precision)
    C = to_host(plan.forward(to_dev(A), to_dev(B)))
    plan.sync()
    if p <= 32:
        ref = _oracle(A, B)
        assert_close(C, ref, REL_TOL, ELEM_TOL, f"{precision} {m}x{n}x{s}x{p}")
    else:
        cols = synth.sample_columns(s, 8)
        ref = _oracle(A, B, cols)
        assert_close(C[:, :, cols], ref, REL_TOL, ELEM_TOL, f"{precision} {m}x{n}x{s}x{p} cols")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_small_workload_full(precision):
    qtp = _qtp()
    A, B = synth.workload("small")
    plan = qtp.Plan(8, 8, 8, 16, precision)
    C = to_host(plan.forward(to_dev(A), to_dev(B)))
    assert_close(C, _oracle(A, B), REL_TOL, ELEM_TOL, "small")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_video_workload_sampled_columns(precision):
    """240x320x64 pixel-like pure quaternion A times 320x240x64 N(0,1) B; 64 sampled columns."""
    qtp = _qtp()
    A, B = synth.workload("video")
    w = synth.WORKLOADS["video"]
    plan = qtp.Plan(w["m"], w["n"], w["s"], w["p"], precision)
    C = to_host(plan.forward(to_dev(A), to_dev(B)))
    plan.sync()
    cols = synth.sample_columns(w["s"], 64)
    ref = _oracle(A, B, cols)
    assert_close(C[:, :, cols], ref, REL_TOL, ELEM_TOL, "video")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_repeated_calls_are_identical(precision):
    qtp = _qtp()
    A, B = _inputs(50, 60, 70, 12, seed=5)
    plan = qtp.Plan(50, 60, 70, 12, precision)
    dA, dB = to_dev(A), to_dev(B)
    C1 = to_host(plan.forward(dA, dB))
    C2 = to_host(plan.forward(dA, dB))
    np.testing.assert_array_equal(C1, C2)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("m,n,s,p", [(5, 4, 3, 1), (6, 9, 7, 4), (12, 10, 14, 7), (33, 17, 40, 32),
                                     (40, 200, 180, 8), (400, 24, 420, 4)])
def test_backward_matches_oracle(precision, m, n, s, p):
    qtp = _qtp()
    A, B = _inputs(m, n, s, p, seed=11 + p)
    G = synth.quat_normal(m, s, p, seed=77 + p)
    plan = qtp.Plan(m, n, s, p, precision)
    dA, dB = plan.backward(to_dev(G), to_dev(A), to_dev(B))
    plan.sync()
    Aq, Bq, Gq = planes_to_comp(A), planes_to_comp(B), planes_to_comp(G)
    assert_close(to_host(dA), Q.tprod_def(Gq, Q.conj_transpose(Bq)), REL_TOL, ELEM_TOL, "dA")
    assert_close(to_host(dB), Q.tprod_def(Q.conj_transpose(Aq), Gq), REL_TOL, ELEM_TOL, "dB")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_backward_single_output(precision):
    qtp = _qtp()
    A, B = _inputs(7, 6, 5, 6, seed=3)
    G = synth.quat_normal(7, 5, 6, seed=4)
    plan = qtp.Plan(7, 6, 5, 6, precision)
    dA, dB = plan.backward(to_dev(G), to_dev(A), to_dev(B), need_dA=False)
    assert dA is None
    Aq, Gq = planes_to_comp(A), planes_to_comp(G)
    assert_close(to_host(dB), Q.tprod_def(Q.conj_transpose(Aq), Gq), REL_TOL, ELEM_TOL, "dB only")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_forward_host_buffers(precision):
    import torch
    qtp = _qtp()
    m, n, s, p = 24, 20, 28, 16
    A, B = _inputs(m, n, s, p, seed=9)
    plan = qtp.Plan(m, n, s, p, precision)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.empty((2, m, s, p, 2), dtype=torch.float32).pin_memory()
    buf = torch.empty(plan.host_buffer_size(), dtype=torch.uint8, device="cuda")
    plan.forward_host(hA, hB, hC, buf)
    plan.sync()
    assert_close(hC.numpy(), _oracle(A, B), REL_TOL, ELEM_TOL, "host buffers")


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape", [(24, 20, 28, 16), (70, 40, 90, 12)])
def test_forward_host_many(precision, shape):
    """Five independent products through qtp_forward_host_many (copies of one
    product overlapping the compute of the previous one): every C equals the
    device-buffer entry point's bit for bit, and the oracle's within
    tolerance; a second call on the same plan and buffer repeats them."""
    import torch
    qtp = _qtp()
    m, n, s, p = shape
    plan = qtp.Plan(m, n, s, p, precision)
    count = 5
    As = [_inputs(m, n, s, p, seed=40 + i) for i in range(count)]
    hA = [torch.from_numpy(a).pin_memory() for a, _ in As]
    hB = [torch.from_numpy(b).pin_memory() for _, b in As]
    hC = [torch.full((2, m, s, p, 2), float("nan")).pin_memory() for _ in range(count)]
    buf = torch.empty(plan.host_many_buffer_size(), dtype=torch.uint8, device="cuda")
    plan.forward_host_many(hA, hB, hC, buf)
    plan.sync()
    for i in range(count):
        ref = plan.forward(hA[i].cuda(), hB[i].cuda())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hC[i].numpy(), ref.cpu().numpy(), err_msg=f"product {i}")
    assert_close(hC[3].numpy(), _oracle(*As[3]), REL_TOL, ELEM_TOL, "host many, product 3")
    first = [c.clone() for c in hC]
    for c in hC:
        c.fill_(float("nan"))
    plan.forward_host_many(hA, hB, hC, buf)
    plan.forward_host_many([], [], [], buf)       # count 0: nothing enqueued
    plan.sync()
    for i in range(count):
        np.testing.assert_array_equal(hC[i].numpy(), first[i].numpy(), err_msg=f"repeat {i}")


def test_forward_host_many_rejects_bad_arguments():
    import ctypes

    import torch
    qtp = _qtp()
    plan = qtp.Plan(8, 8, 8, 8, "bf16x3")
    hA = torch.zeros((2, 8, 8, 8, 2)).pin_memory()
    hC = torch.zeros((2, 8, 8, 8, 2)).pin_memory()
    small = torch.empty(plan.host_many_buffer_size() - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="dev_buffer"):
        plan.forward_host_many([hA], [hA], [hC], small)
    buf = torch.empty(plan.host_many_buffer_size(), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        plan.forward_host_many([hA], [hA, hA], [hC], buf)
    with pytest.raises(ValueError):
        plan.forward_host_many([torch.zeros((2, 8, 8, 4, 2)).pin_memory()], [hA], [hC], buf)
    lib = qtp.lib()
    arr = (ctypes.c_void_p * 1)(hA.data_ptr())
    assert lib.qtp_forward_host_many(plan._h, -1, arr, arr, arr, ctypes.c_void_p(buf.data_ptr()),
                                     buf.numel(), None) == 1
    assert lib.qtp_forward_host_many(plan._h, 1, None, arr, arr, ctypes.c_void_p(buf.data_ptr()),
                                     buf.numel(), None) == 1


# Long tubes: the two-pass lengths 256, 512, 1024 (8-32 tubes per CTA) and
# runtime-radix lengths up to the supported maximum 4096 (one to fifteen
# tubes per CTA), odd and even column counts: sampled entries by
# the definition (O(n p) each) and the whole result against the oracle's FP64
# Algorithm 5.1, itself pinned to the definition on the CPU.
LARGE_P = [(5, 6, 7, 256), (3, 4, 5, 1000), (17, 9, 13, 500), (2, 3, 2, 4096), (4, 6, 5, 2187),
           (6, 5, 7, 512), (3, 4, 5, 1024), (9, 7, 40, 1024)]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("m,n,s,p", LARGE_P)
def test_forward_large_p(precision, m, n, s, p):
    qtp = _qtp()
    A, B = _inputs(m, n, s, p, seed=p + m)
    plan = qtp.Plan(m, n, s, p, precision)
    C = to_host(plan.forward(to_dev(A), to_dev(B)))
    plan.sync()
    Aq, Bq = planes_to_comp(A), planes_to_comp(B)
    assert_close(C, Q.alg51(Aq, Bq), REL_TOL, ELEM_TOL, f"large p={p} vs Alg. 5.1 (FP64)")
    ii, tt, kk = synth.sample_positions(m, s, p, 64)
    ref = Q.tprod_def_entries(Aq, Bq, ii, tt, kk)
    got = planes_to_comp(C)[:, ii, tt, kk]
    assert np.linalg.norm(got - ref) <= REL_TOL * np.linalg.norm(ref), f"large p={p} sampled entries"


@pytest.mark.parametrize("m,n,s,p", LARGE_P[:2])
def test_batched_large_p(m, n, s, p):
    qtp = _qtp()
    shapes = [(m, n, s, p), (m + 1, n, s + 2, p), (4, 4, 4, 8)]
    As = [synth.quat_normal(a, b, q, 70 + i) for i, (a, b, c, q) in enumerate(shapes)]
    Bs = [synth.quat_normal(b, c, q, 80 + i) for i, (a, b, c, q) in enumerate(shapes)]
    plan = qtp.BatchPlan(shapes, "bf16x3")
    Cs = plan.forward([to_dev(a) for a in As], [to_dev(b) for b in Bs])
    plan.sync()
    for i, (a, b, c, q) in enumerate(shapes):
        ref = Q.alg51(planes_to_comp(As[i]), planes_to_comp(Bs[i]))
        assert_close(to_host(Cs[i]), ref, REL_TOL, ELEM_TOL, f"batched product {i} p={q}")


# Products small enough for the one-CTA path (all spectra in shared memory):
# both that path and the three-launch path (QTP_NO_FUSED=1) against the oracle.
FUSED_SHAPES = [(1, 1, 1, 1), (3, 5, 7, 1), (5, 3, 4, 2), (8, 8, 8, 16), (17, 9, 13, 3), (4, 4, 4, 64),
                (8, 3, 5, 31), (4, 12, 9, 12)]


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("m,n,s,p", FUSED_SHAPES)
def test_small_fused_and_staged(fused, precision, m, n, s, p):
    import os
    qtp = _qtp()
    A, B = _inputs(m, n, s, p, seed=3 * m + n + 5 * p)
    if not fused:
        os.environ["QTP_NO_FUSED"] = "1"
    try:
        plan = qtp.Plan(m, n, s, p, precision)
        C = to_host(plan.forward(to_dev(A), to_dev(B)))
        plan.sync()
    finally:
        os.environ.pop("QTP_NO_FUSED", None)
    assert_close(C, _oracle(A, B), REL_TOL, ELEM_TOL, f"{'fused' if fused else 'staged'} {m}x{n}x{s}x{p}")


def test_launch_count_reports_the_route():
    import os
    qtp = _qtp()
    assert qtp.Plan(8, 8, 8, 16, "bf16x3").launch_count() == (1, 5)      # one-CTA route
    assert qtp.Plan(64, 48, 80, 128, "bf16x3").launch_count() == (3, 5)  # Steps 1, 2, 3
    os.environ["QTP_NO_FUSED"] = "1"
    try:
        assert qtp.Plan(8, 8, 8, 16, "fp32").launch_count() == (3, 5)
    finally:
        del os.environ["QTP_NO_FUSED"]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape", [(8, 8, 8, 16), (24, 20, 28, 12), (70, 33, 41, 7), (128, 64, 128, 32)])
def test_backward_from_saved_spectra(precision, shape):
    """qtp_forward_saving + qtp_backward_saved (the spectra of A and B reused)
    give bit for bit the results of qtp_forward + qtp_backward; the first shape
    would take the one-CTA route in qtp_forward, which qtp_forward_saving must
    not take (it writes no spectra)."""
    import torch
    qtp = _qtp()
    m, n, s, p = shape
    A, B = _inputs(m, n, s, p, seed=77)
    dA_np = synth.quat_normal(m, s, p, 78)
    plan = qtp.Plan(m, n, s, p, precision)
    dA_, B_, dC = to_dev(A), to_dev(B), to_dev(dA_np)
    C_ref = plan.forward(dA_, B_)
    gA_ref, gB_ref = plan.backward(dC, dA_, B_)
    C, saved = plan.forward_saving(dA_, B_)
    gA, gB = plan.backward_saved(dC, saved)
    torch.cuda.synchronize()
    if m * n * s * p > 8 * 8 * 8 * 16:
        np.testing.assert_array_equal(to_host(C), to_host(C_ref))
    else:  # qtp_forward took the one-CTA FP32 route, qtp_forward_saving the three steps
        assert_close(to_host(C), _oracle(A, B), REL_TOL, ELEM_TOL, "forward_saving, small product")
    np.testing.assert_array_equal(to_host(gA), to_host(gA_ref))
    np.testing.assert_array_equal(to_host(gB), to_host(gB_ref))
    only_b = plan.backward_saved(dC, saved, need_dA=False)
    torch.cuda.synchronize()
    assert only_b[0] is None
    np.testing.assert_array_equal(to_host(only_b[1]), to_host(gB_ref))


# Every transform form at long tube lengths: the compile-time two-pass form
# (QTP_FFT_SPLIT=2: register DFT-N1 and a tuned two-pass N2 transform; lengths
# it cannot split take the runtime form), the runtime-radix two-pass
# (four-step) form (=1), both through the workspace intermediate and forced
# also for the lengths that have a one-kernel transform, and the one-kernel
# transforms (=0); each against the oracle's FP64 Algorithm 5.1 and sampled
# definition entries.  The plan fixes its form at creation.
@pytest.mark.parametrize("split", ["2", "1", "0"])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("m,n,s,p", [(5, 6, 7, 256), (3, 4, 5, 1000), (9, 7, 40, 1024), (2, 3, 2, 4096),
                                     (7, 5, 6, 243)])
def test_forward_large_p_both_transforms(split, precision, m, n, s, p):
    import os
    qtp = _qtp()
    A, B = _inputs(m, n, s, p, seed=p + 3 * m)
    os.environ["QTP_FFT_SPLIT"] = split
    try:
        plan = qtp.Plan(m, n, s, p, precision)
    finally:
        del os.environ["QTP_FFT_SPLIT"]
    # tensor-core precisions: these small products take the grouped-tile
    # products from p = 256 (one extra launch: the problem record's copy)
    small = 1 if precision != "fp32" and p >= 256 else 0
    assert plan.launch_count()[0] == (3 if split == "0" else 5) + small
    C = to_host(plan.forward(to_dev(A), to_dev(B)))
    plan.sync()
    Aq, Bq = planes_to_comp(A), planes_to_comp(B)
    assert_close(C, Q.alg51(Aq, Bq), REL_TOL, ELEM_TOL, f"p={p} split={split} vs Alg. 5.1 (FP64)")
    ii, tt, kk = synth.sample_positions(m, s, p, 32)
    ref = Q.tprod_def_entries(Aq, Bq, ii, tt, kk)
    got = planes_to_comp(C)[:, ii, tt, kk]
    assert np.linalg.norm(got - ref) <= REL_TOL * np.linalg.norm(ref), f"p={p} split={split} sampled entries"


@pytest.mark.parametrize("split", ["1", None])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("m,n,s,p", [(5, 6, 7, 1000), (4, 3, 5, 4096), (3, 4, 5, 2187)])
def test_backward_large_p(split, precision, m, n, s, p):
    """dA = dC * B^H and dB = A^H * dC at long tube lengths, with the runtime
    two-pass transforms forced in both directions (forward of A, B and dC,
    inverse of dA and dB through the workspace intermediate) and with the
    default choice (the compile-time two-pass form for 1000 = 10 x 100 and
    4096 = 16 x 256; for 2187 = 3^7, which it cannot split, the runtime
    two-pass forward and the one-kernel inverse), against the oracle's FP64
    Algorithm 5.1 on the conjugate transposes."""
    import os
    qtp = _qtp()
    A, B = _inputs(m, n, s, p, seed=p + 1)
    G = synth.quat_normal(m, s, p, seed=p + 2)
    if split is not None:
        os.environ["QTP_FFT_SPLIT"] = split
    try:
        plan = qtp.Plan(m, n, s, p, precision)
    finally:
        os.environ.pop("QTP_FFT_SPLIT", None)
    small = 0 if precision == "fp32" else 1  # the forward's grouped-tile products (backward unchanged)
    if split == "1" or p in (1000, 4096):
        assert plan.launch_count() == (5 + small, 8)
    else:
        assert plan.launch_count() == (4 + small, 7)
    dA, dB = plan.backward(to_dev(G), to_dev(A), to_dev(B))
    plan.sync()
    Aq, Bq, Gq = planes_to_comp(A), planes_to_comp(B), planes_to_comp(G)
    assert_close(to_host(dA), Q.alg51(Gq, Q.conj_transpose(Bq)), REL_TOL, ELEM_TOL, f"dA p={p}")
    assert_close(to_host(dB), Q.alg51(Q.conj_transpose(Aq), Gq), REL_TOL, ELEM_TOL, f"dB p={p}")


# The forward products of small m and s through the grouped kernel (one tile
# per frequency holding both output halves): taken by itself from p = 256,
# forced here (QTP_SMALL_TILES=1) at short tube lengths too.  Plain and
# transposed tiles (the larger of m and s on the 128 rows), ragged K up to the
# single-accumulator limit, both tensor-core precisions, and a second call with
# other buffers (the tensor maps encoded again) against the oracle.
@pytest.mark.parametrize("precision", ["bf16x3", "bf16"])
@pytest.mark.parametrize("m,n,s,p,env", [(64, 64, 64, 16, "1"), (128, 40, 64, 8, "1"), (40, 30, 128, 12, "1"),
                                         (100, 384, 50, 5, "1"), (33, 20, 17, 300, None)])
def test_forward_small_tiles_route(precision, m, n, s, p, env):
    import os
    import torch
    qtp = _qtp()
    if env is not None:
        os.environ["QTP_SMALL_TILES"] = env
    try:
        plan = qtp.Plan(m, n, s, p, precision)
        os.environ["QTP_SMALL_TILES"] = "0"  # the single-product kernel, for comparison
        plan_tc = qtp.Plan(m, n, s, p, precision)
    finally:
        os.environ.pop("QTP_SMALL_TILES", None)
    assert plan.launch_count()[0] == plan_tc.launch_count()[0] + 1
    for call in range(2):
        A, B = _inputs(m, n, s, p, seed=7 * call + p + m)
        dA, dB = to_dev(A), to_dev(B)
        C = to_host(plan.forward(dA, dB))
        plan.sync()
        C_tc = to_host(plan_tc.forward(dA, dB))
        plan_tc.sync()
        Aq, Bq = planes_to_comp(A), planes_to_comp(B)
        ref = Q.alg51(Aq, Bq)
        if precision == "bf16x3":
            assert_close(C, ref, REL_TOL, ELEM_TOL, f"grouped tiles, call {call}")
        else:  # one bf16 product: the single-product kernel's error level, not more
            err = np.linalg.norm(planes_to_comp(C) - ref) / np.linalg.norm(ref)
            err_tc = np.linalg.norm(planes_to_comp(C_tc) - ref) / np.linalg.norm(ref)
            assert err <= 1.5 * err_tc + 1e-6, (err, err_tc)
        del dA, dB
        torch.cuda.synchronize()
