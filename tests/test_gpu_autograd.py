"""Differentiation through libqtp's hand-written backward (torch.autograd.Function).

Workload: loss = ||A*B - T||_F^2 with A 128x64x32, B 64x128x32, T 128x128x32,
N(0,1) components, FP32.  dA = dC*B^H and dB = A^H*dC come from qtp_backward.
Checks: the oracle's definition-based gradient; central finite differences
(h = 1e-3) evaluated in FP64 by the oracle on 64 entries of A and of B and on 8
random joint directions; 200 gradient-descent steps of a low-tubal-rank
factorisation whose first 10 steps match an FP64 replay, with a checkpoint /
resume that reproduces the uninterrupted run exactly.
"""
import io

import numpy as np
import pytest

import oracle as Q
from paper_2212_14318_gb300 import synth
from tests._gpu import rel_fro, to_dev, to_host
from tests._qlayout import planes_to_comp

pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["diff"]
M, N, S, P = W["m"], W["n"], W["s"], W["p"]


def _inputs():
    A, B = synth.workload("diff")
    return A, B, synth.target("diff")


def _loss_and_grads(A, B, T, precision):
    import torch
    from paper_2212_14318_gb300.autograd import tprod
    a = to_dev(A).requires_grad_(True)
    b = to_dev(B).requires_grad_(True)
    t = to_dev(T)
    loss = ((tprod(a, b, precision) - t) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    return float(loss.item()), to_host(a.grad), to_host(b.grad)


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_autograd_matches_oracle_gradient(precision):
    A, B, T = _inputs()
    Aq, Bq, Tq = planes_to_comp(A), planes_to_comp(B), planes_to_comp(T)
    loss, gA, gB = _loss_and_grads(A, B, T, precision)
    dA, dB = Q.grad_def(Aq, Bq, Tq)
    assert rel_fro(planes_to_comp(gA), dA) <= 1e-5
    assert rel_fro(planes_to_comp(gB), dB) <= 1e-5
    assert abs(loss - Q.loss_def(Aq, Bq, Tq)) <= 1e-5 * Q.loss_def(Aq, Bq, Tq)


def test_gradient_matches_central_differences_fp64():
    A, B, T = _inputs()
    Aq, Bq, Tq = planes_to_comp(A), planes_to_comp(B), planes_to_comp(T)
    _, gA, gB = _loss_and_grads(A, B, T, "bf16x3")
    gA, gB = planes_to_comp(gA), planes_to_comp(gB)
    rng = np.random.default_rng(31)
    h = 1e-3
    fd, an = [], []
    for _ in range(64):   # entries of A: only row i of C moves
        c, i, j, r = (int(rng.integers(0, d)) for d in Aq.shape)
        rows = []
        for sgn in (1, -1):
            Ai = Aq[:, i:i + 1].copy()
            Ai[c, 0, j, r] += sgn * h
            rows.append(np.sum((Q.tprod_def(Ai, Bq) - Tq[:, i:i + 1]) ** 2))
        fd.append((rows[0] - rows[1]) / (2 * h))
        an.append(gA[c, i, j, r])
    for _ in range(64):   # entries of B: only column t of C moves
        c, j, t, r = (int(rng.integers(0, d)) for d in Bq.shape)
        cols = []
        for sgn in (1, -1):
            Bt = Bq.copy()
            Bt[c, j, t, r] += sgn * h
            cols.append(np.sum((Q.tprod_def_columns(Aq, Bt, [t]) - Tq[:, :, t:t + 1]) ** 2))
        fd.append((cols[0] - cols[1]) / (2 * h))
        an.append(gB[c, j, t, r])
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) <= 1e-5 * np.linalg.norm(fd)
    for _ in range(8):    # joint directions: the loss is quartic along them, FD error O(h^2)
        VA = rng.standard_normal(Aq.shape)
        VB = rng.standard_normal(Bq.shape)
        lp = np.sum((Q.alg51(Aq + h * VA, Bq + h * VB) - Tq) ** 2)
        lm = np.sum((Q.alg51(Aq - h * VA, Bq - h * VB) - Tq) ** 2)
        d_fd = (lp - lm) / (2 * h)
        d_an = float(np.sum(gA * VA) + np.sum(gB * VB))
        assert abs(d_fd - d_an) <= 1e-4 * abs(d_fd)


def _step_size(Aq, Bq):
    """0.5 / L with L = 2 max(||bcirc(A)||^2, ||bcirc(B)||^2), by 20 power iterations (FP64 oracle)."""
    rng = np.random.default_rng(32)

    def top(op, shape):
        v = rng.standard_normal(shape)
        for _ in range(20):
            v = op(v)
            v /= np.linalg.norm(v)
        return float(np.sum(v * op(v)))
    lb = top(lambda X: Q.alg51(Q.alg51(X, Bq), Q.conj_transpose(Bq)), (4, 4, N, P))
    la = top(lambda X: Q.alg51(Q.conj_transpose(Aq), Q.alg51(Aq, X)), (4, N, 4, P))
    return 0.5 / (2.0 * max(la, lb))


def test_low_tubal_rank_factorisation_200_steps_with_replay_and_resume():
    """Gradient descent on ||A*B - T||^2 (tubal rank <= 64 of a 128 x 128 target),
    bounded below by the truncated T-SVD of T."""
    import torch
    from paper_2212_14318_gb300.autograd import tprod
    rng = np.random.default_rng(33)
    T = synth.target("diff").astype(np.float64)
    scale = (1.0 / (4 * N * P)) ** 0.25          # A*B starts at the magnitude of T
    A0 = (rng.standard_normal((2, M, N, P, 2)) * scale).astype(np.float32)
    B0 = (rng.standard_normal((2, N, S, P, 2)) * scale).astype(np.float32)
    Tq = planes_to_comp(T)
    eta = _step_size(planes_to_comp(A0), planes_to_comp(B0))

    def run(a, b, steps, losses=None, snapshots=None):
        t = to_dev(T.astype(np.float32))
        for k in range(steps):
            a.grad = None
            b.grad = None
            loss = ((tprod(a, b, "bf16x3") - t) ** 2).sum()
            loss.backward()
            with torch.no_grad():
                a -= eta * a.grad
                b -= eta * b.grad
            if losses is not None:
                losses.append(float(loss.item()))
            if snapshots is not None and k < 10:
                snapshots.append((to_host(a), to_host(b)))
        return a, b

    a = to_dev(A0).requires_grad_(True)
    b = to_dev(B0).requires_grad_(True)
    losses, snaps = [], []
    a, b = run(a, b, 200, losses, snaps)
    losses = np.array(losses)
    assert np.all(np.diff(losses) <= 1e-6 * losses[:-1]), "loss increased"
    assert losses[-1] < 0.75 * losses[0]
    # A*B has tubal rank <= 64, so by Eckart-Young on every M_f (and Parseval)
    # no step can go below the truncated T-SVD of T (FP64 oracle); the descent
    # gets within 1% of it in 200 steps (FP64 replay: 1.008)
    from oracle import tsvd as TS
    best = TS.truncation_error_sq(TS.tsvd(Tq)[3], N)
    assert losses[-1] >= best * (1 - 1e-4), (losses[-1], best)
    assert losses[-1] <= 1.03 * best, losses[-1] / best

    # FP64 replay of the first 10 steps with oracle gradients
    Aq, Bq = planes_to_comp(A0), planes_to_comp(B0)
    for k in range(10):
        R = 2.0 * (Q.alg51(Aq, Bq) - Tq)
        dA = Q.alg51(R, Q.conj_transpose(Bq))
        dB = Q.alg51(Q.conj_transpose(Aq), R)
        Aq, Bq = Aq - eta * dA, Bq - eta * dB
        ga, gb = snaps[k]
        assert rel_fro(planes_to_comp(ga), Aq) <= 1e-4, k
        assert rel_fro(planes_to_comp(gb), Bq) <= 1e-4, k

    # checkpoint after 100 steps, resume, and reproduce the uninterrupted run bit for bit
    a2 = to_dev(A0).requires_grad_(True)
    b2 = to_dev(B0).requires_grad_(True)
    a2, b2 = run(a2, b2, 100)
    buf = io.BytesIO()
    torch.save({"A": a2.detach().cpu(), "B": b2.detach().cpu(), "step": 100}, buf)
    buf.seek(0)
    state = torch.load(buf)
    a3 = state["A"].cuda().requires_grad_(True)
    b3 = state["B"].cuda().requires_grad_(True)
    a3, b3 = run(a3, b3, 100)
    np.testing.assert_array_equal(to_host(a3), to_host(a))
    np.testing.assert_array_equal(to_host(b3), to_host(b))
