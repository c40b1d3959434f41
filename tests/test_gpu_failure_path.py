"""The bounded-wait failure path of the tensor-core products, made to run.

Every mbarrier wait in the products kernels is bounded; on expiry the kernel
records a code in the plan's device error word, waits (bounded) for its own
copies and MMAs in flight, frees its tensor memory and returns, and the next
qtp_plan_sync / qtp_batch_plan_sync reports QTP_ERR_TIMEOUT.  Here the failure
is made on the host: QTP_INJECT_WITHHOLD=k tells the operand producer never to
load K step k (a dependency that nothing satisfies) and QTP_INJECT_WAIT_NS
shortens every wait of those launches to a few milliseconds.  No address
outside the kernels' buffers is touched and nothing traps; afterwards a normal
call on the same plan must match the FP64 oracle, which shows the context is
still usable.
"""
import os

import pytest

import oracle as Q
from paper_2212_14318_gb300 import synth
from tests._gpu import assert_close, to_dev, to_host
from tests._qlayout import planes_to_comp

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
ELEM_TOL = 1e-4
QTP_ERR_TIMEOUT = 5


class _Withheld:
    def __init__(self, k, wait_ns=5_000_000):
        self.k, self.wait_ns = k, wait_ns

    def __enter__(self):
        os.environ["QTP_INJECT_WITHHOLD"] = str(self.k)
        os.environ["QTP_INJECT_WAIT_NS"] = str(self.wait_ns)

    def __exit__(self, *exc):
        os.environ.pop("QTP_INJECT_WITHHOLD", None)
        os.environ.pop("QTP_INJECT_WAIT_NS", None)


def _qtp():
    import torch
    from paper_2212_14318_gb300 import qtp
    assert torch.cuda.is_available()
    return qtp


# (m, n, s, p, withheld K step): one accumulator pair (6 K steps); promoted
# accumulators, the step withheld after the first promotion (segments of 32)
@pytest.mark.parametrize("m,n,s,p,k", [(64, 48, 80, 8, 3), (40, 1200, 36, 2, 40)])
def test_forward_wait_expires_then_plan_recovers(m, n, s, p, k):
    qtp = _qtp()
    A = synth.quat_normal(m, n, p, seed=90)
    B = synth.quat_normal(n, s, p, seed=91)
    dA, dB = to_dev(A), to_dev(B)
    plan = qtp.Plan(m, n, s, p, "bf16x3")
    with _Withheld(k):
        plan.forward(dA, dB)
        with pytest.raises(qtp.QtpError) as exc:
            plan.sync()
    assert exc.value.status == QTP_ERR_TIMEOUT
    assert "gave up" in str(exc.value)
    plan.sync()  # the error word was cleared by the report
    C = to_host(plan.forward(dA, dB))
    plan.sync()
    assert_close(C, Q.tprod_def(planes_to_comp(A), planes_to_comp(B)), REL_TOL, ELEM_TOL, "after recovery")


def test_batched_wait_expires_then_plan_recovers():
    qtp = _qtp()
    shapes = [(40, 30, 50, 8), (16, 20, 24, 12), (130, 24, 30, 4)]
    As = [synth.quat_normal(a, b, q, 95 + i) for i, (a, b, c, q) in enumerate(shapes)]
    Bs = [synth.quat_normal(b, c, q, 97 + i) for i, (a, b, c, q) in enumerate(shapes)]
    dA, dB = [to_dev(a) for a in As], [to_dev(b) for b in Bs]
    plan = qtp.BatchPlan(shapes, "bf16x3", graph=False)
    with _Withheld(2):
        Cs = plan.forward(dA, dB)
        with pytest.raises(qtp.QtpError) as exc:
            plan.sync()
    assert exc.value.status == QTP_ERR_TIMEOUT
    plan.forward(dA, dB, Cs)
    plan.sync()
    for i in range(len(shapes)):
        ref = Q.tprod_def(planes_to_comp(As[i]), planes_to_comp(Bs[i]))
        assert_close(to_host(Cs[i]), ref, REL_TOL, ELEM_TOL, f"batched product {i} after recovery")
