"""Pins of the FP64 T-SVD oracle (``oracle.tsvd``).

Every property is checked with arithmetic the T-SVD does not use: the
T-product and conjugate transpose by their definitions (``tprod_def``,
``conj_transpose``: slice sums of Hamilton products, no FFT), the quaternion
matrix product for p = 1, numpy's SVD of real FFT slices for the real special
case, and Parseval's identity.
"""
import numpy as np
import pytest

import oracle as Q
from oracle import tsvd as T

SHAPES = [(3, 4, 5), (4, 3, 6), (2, 2, 1), (5, 5, 8), (1, 3, 4), (3, 1, 2), (4, 6, 7), (6, 4, 2)]


def rand(rng, m, n, p):
    return rng.standard_normal((4, m, n, p))


def eye_tensor(k, p):
    return Q.identity(k, p)


def tp(*xs):
    acc = xs[0]
    for x in xs[1:]:
        acc = Q.tprod_def(acc, x)
    return acc


def reconstruct(U, S, V):
    return tp(U, S, Q.conj_transpose(V))


@pytest.mark.parametrize("m,n,p", SHAPES)
def test_structure_of_the_spectral_matrices(m, n, p):
    """M_f(A * B) = M_f(A) M_f(B), M_f(A^H) = M_f(A)^H, M_(-f)(A) = Q conj(M_f) Q^T."""
    rng = np.random.default_rng(10 + m + 10 * n + 100 * p)
    A, B = rand(rng, m, n, p), rand(rng, n, 3, p)
    C = Q.tprod_def(A, B)
    AH = Q.conj_transpose(A)
    for f in range(p):
        g = (-f) % p
        Mf = T.spectral_matrix(A, f)
        np.testing.assert_allclose(T.spectral_matrix(C, f), Mf @ T.spectral_matrix(B, f), atol=1e-11)
        np.testing.assert_allclose(T.spectral_matrix(AH, f), Mf.conj().T, atol=1e-12)
        np.testing.assert_allclose(T.spectral_matrix(A, g), T._Q(m) @ np.conj(Mf) @ T._Q(n).T, atol=1e-12)


@pytest.mark.parametrize("m,n,p", SHAPES)
def test_tsvd_reconstructs_orthogonal_f_diagonal(m, n, p):
    rng = np.random.default_rng(20 + m + 10 * n + 100 * p)
    A = rand(rng, m, n, p)
    U, S, V, sigma = T.tsvd(A)
    k = min(m, n)
    assert U.shape == (4, m, k, p) and S.shape == (4, k, k, p) and V.shape == (4, n, k, p)
    np.testing.assert_allclose(reconstruct(U, S, V), A, atol=1e-11)
    np.testing.assert_allclose(tp(Q.conj_transpose(U), U), eye_tensor(k, p), atol=1e-12)
    np.testing.assert_allclose(tp(Q.conj_transpose(V), V), eye_tensor(k, p), atol=1e-12)
    off = ~np.eye(k, dtype=bool)
    assert np.all(S[:, off, :] == 0) and np.all(S[2:] == 0)      # f-diagonal, no j part
    assert np.all(sigma >= 0)
    assert np.all(np.diff(sigma, axis=1) <= 1e-12)               # each spectrum sorted


@pytest.mark.parametrize("m,n,p", SHAPES)
def test_parseval_and_truncation_closed_form(m, n, p):
    rng = np.random.default_rng(30 + m + 10 * n + 100 * p)
    A = rand(rng, m, n, p)
    U, S, V, sigma = T.tsvd(A)
    np.testing.assert_allclose(np.sum(A * A), np.sum(sigma ** 2) / p, rtol=1e-12)
    for r in range(min(m, n) + 1):
        Ar = reconstruct(*T.truncate(U, S, V, r)) if r > 0 else np.zeros_like(A)
        np.testing.assert_allclose(np.sum((A - Ar) ** 2), T.truncation_error_sq(sigma, r), rtol=1e-9, atol=1e-12)


def test_truncation_beats_perturbed_competitors():
    """Eckart-Young in the T-product sense: nearby tubal-rank-r tensors
    (perturbed factors) never approximate A better than the truncated T-SVD."""
    rng = np.random.default_rng(40)
    m, n, p, r = 5, 4, 6, 2
    A = rand(rng, m, n, p)
    U, S, V, sigma = T.tsvd(A)
    Ur, Sr, Vr = T.truncate(U, S, V, r)
    best = np.sum((A - reconstruct(Ur, Sr, Vr)) ** 2)
    for eps in (1e-1, 1e-2, 1e-3):
        for _ in range(10):
            X = Ur + eps * rng.standard_normal(Ur.shape)
            Y = tp(Sr, Q.conj_transpose(Vr)) + eps * rng.standard_normal((4, r, n, p))
            assert np.sum((A - tp(X, Y)) ** 2) >= best * (1 - 1e-12)


@pytest.mark.parametrize("m,n,p", [(4, 3, 6), (3, 5, 7), (4, 4, 1)])
def test_real_special_case_is_the_real_t_svd(m, n, p):
    """b = c = d = 0: every spectrum is the singular values of the FFT slice
    (the real t-SVD of Kilmer and Martin), numpy's SVD."""
    rng = np.random.default_rng(50 + p)
    A = np.zeros((4, m, n, p))
    A[0] = rng.standard_normal((m, n, p))
    _, _, _, sigma = T.tsvd(A)
    Ah = np.fft.fft(A[0], axis=-1)
    for f in range(p):
        np.testing.assert_allclose(sigma[f], np.linalg.svd(Ah[..., f], compute_uv=False), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("m,n", [(3, 4), (4, 2), (3, 3)])
def test_p1_is_the_quaternion_matrix_svd(m, n):
    """p = 1: a quaternion matrix SVD A = U S V^H with the quaternion matrix
    product (Hamilton arithmetic), and the complex adjoint's singular values
    are sigma, each twice."""
    rng = np.random.default_rng(60 + m + n)
    A = rand(rng, m, n, 1)
    U, S, V, sigma = T.tsvd(A)
    u, s_, v = U[..., 0], S[..., 0], V[..., 0]
    np.testing.assert_allclose(Q.qmatmul(Q.qmatmul(u, s_), Q.qmat_conj_transpose(v)), A[..., 0], atol=1e-12)
    np.testing.assert_allclose(Q.qmatmul(Q.qmat_conj_transpose(u), u)[0], np.eye(min(m, n)), atol=1e-12)
    A1, A2 = A[0, ..., 0] + 1j * A[1, ..., 0], A[2, ..., 0] + 1j * A[3, ..., 0]
    chi = np.block([[A1, A2], [-np.conj(A2), np.conj(A1)]])
    sv = np.linalg.svd(chi, compute_uv=False)
    np.testing.assert_allclose(np.repeat(sigma[0], 2), sv[:2 * min(m, n)], rtol=1e-11)


@pytest.mark.parametrize("p", [1, 4, 5])
def test_rank_deficient_inputs(p):
    """The zero tensor and a tubal-rank-1 tensor: the factors stay unitary,
    the spectra vanish beyond the rank, the product is rebuilt."""
    rng = np.random.default_rng(70 + p)
    m, n = 4, 3
    for A in (np.zeros((4, m, n, p)), tp(rand(rng, m, 1, p), Q.conj_transpose(rand(rng, n, 1, p)))):
        U, S, V, sigma = T.tsvd(A)
        np.testing.assert_allclose(reconstruct(U, S, V), A, atol=1e-11)
        np.testing.assert_allclose(tp(Q.conj_transpose(U), U), eye_tensor(n, p), atol=1e-10)
        np.testing.assert_allclose(tp(Q.conj_transpose(V), V), eye_tensor(n, p), atol=1e-10)
        np.testing.assert_allclose(sigma[:, 1:], 0, atol=1e-10)


def test_self_paired_frequency_needs_the_partner_structure():
    """At f = 0 = -f the odd/even split of the other frequencies is not a
    valid factor: the two block readings of U2(0) it implies disagree, which
    is why the oracle takes W's second half as the partners of the first."""
    rng = np.random.default_rng(80)
    A = rand(rng, 3, 3, 4)
    M = T.spectral_matrix(A, 0)
    W, s, _ = np.linalg.svd(M, full_matrices=False)
    Wa, Wb = W[:, 0::2], W[:, 1::2]                  # the f != g split, wrong here
    U1, U2 = Wa[:3], Wb[:3]
    bad_U2_at_g = -np.conj(Wa[3:])                   # what U2(0) must also equal
    assert np.max(np.abs(U2 - bad_U2_at_g)) > 1e-3   # the two readings of U2(0) disagree
