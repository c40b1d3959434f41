"""T-SVD through the C ABI (qtp_tsvd) against the FP64 oracle (oracle.tsvd).

The singular vectors are not unique (phases, equal singular values), so the
tests compare what is: sigma element by element, and check the rest for
validity with FP64 arithmetic on the returned factors: A = U * S * V^H,
U^H * U = V^H * V = I, S exactly f-diagonal, the truncation error by
Parseval.  Tolerances: the Jacobi sweeps stop rotating a column pair once
|x^H y| <= 2e-6 |x| |y| (FP32), so orthogonality holds to a few 1e-6;
reconstruction and sigma to FP32 rounding of the accumulated rotations.
"""
import numpy as np
import pytest

import oracle as Q
from oracle import tsvd as T
from paper_2212_14318_gb300 import synth
from tests._gpu import to_dev, to_host
from tests._qlayout import planes_to_comp

pytestmark = pytest.mark.gpu

# (m, n, p): square, tall (sweeps on M_f) and wide (on M_f^H); self-paired
# frequencies (p = 1, even p); odd and prime p; k = 64 (the maximum, global
# scratch); a tall shape whose pair matrices still fit in shared memory.
SHAPES = [(1, 1, 1), (5, 3, 1), (3, 5, 2), (8, 8, 8), (16, 12, 16), (12, 16, 12), (40, 24, 31), (24, 40, 7),
          (64, 64, 32), (200, 16, 8), (16, 300, 5), (130, 20, 100),
          # columns in registers handed over between warps (2 max(m, n) <= 256 with the buffers in the
          # global scratch): 32, 40 and 40 pair slots, so CTAs with idle warps at most cluster sizes; the
          # wide input (sweeps on M_f^H); test_tsvd_ring_cluster_counts runs them at fixed cluster sizes
          (128, 32, 4), (120, 40, 6), (40, 120, 9),
          # sweeps from L2 with the register pair step (256 < 2 max(m, n) <= 512, buffers above 200 KB)
          (200, 64, 8)]
SIGMA_TOL = 2e-5     # relative to the largest singular value
REC_TOL = 1e-5       # relative Frobenius error of U * S * V^H
ORTH_TOL = 2e-5      # max |U^H * U - I| entry


def tp(X, Y):
    """T-product in FP64 by the oracle's Algorithm 5.1 (pinned to the definition)."""
    return Q.alg51(X, Y)


def factors(m, n, p, seed):
    from paper_2212_14318_gb300 import qtp
    A = synth.quat_normal(m, n, p, seed)
    U, S, V, sigma = qtp.tsvd(to_dev(A), check=True)  # every pair's sweeps converged (qtp_tsvd_sync)
    return (planes_to_comp(A), planes_to_comp(to_host(U)), planes_to_comp(to_host(S)),
            planes_to_comp(to_host(V)), to_host(sigma).astype(np.float64))


def check_valid(Aq, U, S, V, sigma, tag):
    m, n, p = Aq.shape[1:]
    k = min(m, n)
    rec = tp(tp(U, S), Q.conj_transpose(V))
    assert Q.rel_fro(rec, Aq) <= REC_TOL, (tag, Q.rel_fro(rec, Aq))
    for X in (U, V):
        G = tp(Q.conj_transpose(X), X)
        assert np.max(np.abs(G - Q.identity(k, p))) <= ORTH_TOL, (tag, np.max(np.abs(G - Q.identity(k, p))))
    off = ~np.eye(k, dtype=bool)
    assert np.all(S[:, off, :] == 0) and np.all(S[2:] == 0), tag
    assert np.all(sigma >= 0) and np.all(np.diff(sigma, axis=1) <= 1e-6 * max(sigma.max(), 1e-30)), tag


@pytest.mark.parametrize("m,n,p", SHAPES)
def test_tsvd_matches_oracle(m, n, p):
    Aq, U, S, V, sigma = factors(m, n, p, seed=300 + m + 7 * n + 13 * p)
    _, _, _, sref = T.tsvd(Aq)
    assert np.max(np.abs(sigma - sref)) <= SIGMA_TOL * sref.max(), np.max(np.abs(sigma - sref)) / sref.max()
    check_valid(Aq, U, S, V, sigma, (m, n, p))


@pytest.mark.parametrize("m,n,p", [(8, 6, 5), (12, 16, 4)])
def test_tsvd_truncation_error(m, n, p):
    """||A - U_r * S_r * V_r^H||^2 = (1 / p) sum of the dropped sigma^2 (Parseval)."""
    Aq, U, S, V, sigma = factors(m, n, p, seed=700 + p)
    total = np.sum(Aq * Aq)
    for r in range(min(m, n) + 1):
        if r == 0:
            err = total
        else:
            Ur, Sr, Vr = T.truncate(U, S, V, r)
            err = np.sum((Aq - tp(tp(Ur, Sr), Q.conj_transpose(Vr))) ** 2)
        assert abs(err - T.truncation_error_sq(sigma, r)) <= 2e-5 * total, (r, err, T.truncation_error_sq(sigma, r))


@pytest.mark.parametrize("m,n", [(8, 6), (128, 32)])
@pytest.mark.parametrize("p", [1, 4, 5])
def test_tsvd_rank_deficient(m, n, p):
    """The zero tensor and a tubal-rank-1 tensor: unitary factors (null
    columns completed), spectra zero beyond the rank, the tensor rebuilt.
    8 x 6 runs in one CTA's shared memory; 128 x 32 in a cluster with the
    global scratch, where the self-paired frequencies fall back from the
    one-step structured completion (null candidates) to the sequential one."""
    import torch
    from paper_2212_14318_gb300 import qtp
    from tests._qlayout import comp_to_planes
    rng = np.random.default_rng(90 + p)
    x, y = rng.standard_normal((4, m, 1, p)), rng.standard_normal((4, n, 1, p))
    for Aq in (np.zeros((4, m, n, p)), Q.tprod_def(x, Q.conj_transpose(y))):
        A = comp_to_planes(Aq).astype(np.float32)
        U, S, V, sigma = qtp.tsvd(to_dev(A), check=True)  # every pair's sweeps converged (qtp_tsvd_sync)
        torch.cuda.synchronize()
        U, S, V = (planes_to_comp(to_host(t)) for t in (U, S, V))
        sigma = to_host(sigma).astype(np.float64)
        k = min(m, n)
        for X in (U, V):
            G = tp(Q.conj_transpose(X), X)
            assert np.max(np.abs(G - Q.identity(k, p))) <= ORTH_TOL
        scale = max(np.sqrt(np.sum(Aq * Aq)), 1.0)
        assert np.max(sigma[:, 1:]) <= 1e-5 * scale
        rec = tp(tp(U, S), Q.conj_transpose(V))
        assert np.sqrt(np.sum((rec - Aq) ** 2)) <= 1e-5 * scale


@pytest.mark.parametrize("m,n,p,counts", [(128, 32, 4, (2, 3, 5, 8)), (120, 40, 6, (3, 4, 7)),
                                           (40, 120, 9, (3, 6)), (64, 64, 32, (4, 5, 8))])
def test_tsvd_ring_cluster_counts(m, n, p, counts, monkeypatch):
    """The register ring's pair slots spread over any count of CTAs from the
    smallest that holds them (QTP_TSVD_CLUSTER fixes it; by default the
    launch takes the count from the cluster occupancy): the rotations, their
    order and every other step's arithmetic are the same, so the factors are
    bit-identical to the default count's, which are valid against the
    oracle.  8 CTAs for 17 pairs runs two waves of clusters."""
    from paper_2212_14318_gb300 import qtp
    A = synth.quat_normal(m, n, p, 11)
    Ad = to_dev(A)
    monkeypatch.delenv("QTP_TSVD_CLUSTER", raising=False)
    ref = [to_host(t) for t in qtp.tsvd(Ad, check=True)]
    for c in counts:
        monkeypatch.setenv("QTP_TSVD_CLUSTER", str(c))
        out = [to_host(t) for t in qtp.tsvd(Ad, check=True)]
        for a, b in zip(ref, out):
            np.testing.assert_array_equal(a, b, err_msg=f"{c} CTAs")
    U, S, V = (planes_to_comp(t) for t in ref[:3])
    sigma = ref[3].astype(np.float64)
    Aq = planes_to_comp(A)
    _, _, _, sref = T.tsvd(Aq)
    assert np.max(np.abs(sigma - sref)) <= SIGMA_TOL * sref.max()
    check_valid(Aq, U, S, V, sigma, (m, n, p))


def test_tsvd_repeatable():
    from paper_2212_14318_gb300 import qtp
    A = to_dev(synth.quat_normal(24, 16, 12, 5))
    r1 = [to_host(t) for t in qtp.tsvd(A)]
    r2 = [to_host(t) for t in qtp.tsvd(A)]
    for a, b in zip(r1, r2):
        np.testing.assert_array_equal(a, b)
