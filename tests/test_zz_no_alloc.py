"""qtp_forward_noalloc against the FP64 oracle and against qtp_forward.

qtp_forward_noalloc serves callers that may not allocate device memory (their
memory belongs to another allocator, or cudaMalloc's synchronisation is too
costly): it takes no plan and no workspace and keeps its scratch in a static
device array inside the library.  This file is collected last so that a run
stopping at the first failure has run every other test before it; it also
passes alone in a fresh process.
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


def _lib():
    import torch
    from paper_2212_14318_gb300 import build, qtp
    assert torch.cuda.is_available()
    build.build()
    return qtp


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_noalloc_matches_forward_on_two_calls_in_a_row(precision):
    qtp = _lib()
    # two consecutive calls with different shapes and p: the second call must
    # not see the first call's twiddles or error word
    # (a third call at a long tube length: the transform's workspace intermediate
    # and its second twiddle table also live in the static array)
    for call, (m, n, s, p) in enumerate([(40, 24, 36, 64), (17, 9, 13, 12), (5, 4, 6, 1000)]):
        A = synth.quat_normal(m, n, p, seed=500 + call)
        B = synth.quat_normal(n, s, p, seed=600 + call)
        dA, dB = to_dev(A), to_dev(B)
        ref = qtp.Plan(m, n, s, p, precision).forward(dA, dB)
        got = to_host(qtp.forward_noalloc(dA, dB, precision=precision))
        # the definition (Definition 2.3, FP64; through the oracle's FP64 Algorithm 5.1,
        # pinned to it, at the long tube length), as every parity test
        Aq, Bq = planes_to_comp(A), planes_to_comp(B)
        ref_def = Q.tprod_def(Aq, Bq) if p <= 64 else Q.alg51(Aq, Bq)
        assert_close(got, ref_def, REL_TOL, ELEM_TOL, f"noalloc call {call} {precision} vs oracle")
        # and the entry point that allocates, on the same device inputs
        assert_close(got, planes_to_comp(to_host(ref)), REL_TOL, ELEM_TOL,
                     f"noalloc call {call} {precision} vs qtp_forward")


def test_noalloc_rejects_products_beyond_the_static_array():
    import ctypes
    import torch
    qtp = _lib()
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    st = qtp.lib().qtp_forward_noalloc(1024, 1024, 1024, 128, 1, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None)
    assert st == 3  # QTP_ERR_WORKSPACE, rejected on the host before any launch
    assert b"static array" in qtp.lib().qtp_last_error()
