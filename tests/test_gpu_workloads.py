"""Full-size workloads through the C ABI, checked against the FP64 oracle on
sampled outputs it computes one by one (mode-1 fibres C(:, t, k) by the
definition)."""
import numpy as np
import pytest

import oracle as Q
from paper_2212_14318_gb300 import synth
from tests._gpu import assert_close, rel_fro, to_dev
from tests._qlayout import planes_to_comp

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
ELEM_TOL = 1e-4


def _fibres(C_dev, tt, kk):
    """Gather C(:, t, k) for the sampled pairs on the device, return plane layout (2, m, P, 2)."""
    import torch
    t = torch.as_tensor(tt, device=C_dev.device)
    k = torch.as_tensor(kk, device=C_dev.device)
    return C_dev[:, :, t, k, :].cpu().numpy().astype(np.float64)


def test_precision_workload_split_bf16_vs_fp32_vs_bf16():
    """1024 x 1024 x 128 quaternion tensors, N(0,1): split-BF16 and FP32 products
    both within 1e-5 of the oracle on 128 sampled fibres; BF16-only is worse."""
    from paper_2212_14318_gb300 import qtp
    w = synth.WORKLOADS["precision"]
    m, n, s, p = w["m"], w["n"], w["s"], w["p"]
    A, B = synth.workload("precision")
    dA, dB = to_dev(A), to_dev(B)
    rng = np.random.default_rng(synth.SEED_SAMPLE)
    tt, kk = rng.integers(0, s, 128), rng.integers(0, p, 128)
    Aq = planes_to_comp(A)
    del A
    ref = Q.tprod_def_pairs(Aq, planes_to_comp(B), tt, kk)          # (4, m, 128)
    del Aq
    errs = {}
    for precision in ("bf16x3", "fp32", "bf16"):
        plan = qtp.Plan(m, n, s, p, precision)
        C = plan.forward(dA, dB)
        plan.sync()
        got = _fibres(C, tt, kk)                                       # (2, m, 128, 2)
        errs[precision] = rel_fro(planes_to_comp(got), ref)
        if precision != "bf16":
            assert_close(got, ref, REL_TOL, ELEM_TOL, f"precision workload {precision}")
        del C, plan
    assert errs["bf16"] > 10 * errs["bf16x3"], errs
    print("relative errors vs FP64 oracle:", errs)
