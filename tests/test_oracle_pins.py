"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

None of these compares the oracle with itself: each check uses an independent
route (the complex-adjoint representation, numpy's FFT, explicit bcirc
matrices, pure-Python loops, algebraic invariants, finite differences) or a
value printed in the paper (tests/golden/).
"""
import json
import os

import numpy as np
import pytest

import oracle as Q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
UNITS = {"1": 0, "i": 1, "j": 2, "k": 3}


def rand_q(rng, *shape):
    return rng.standard_normal((4,) + shape)


def chi(X):
    """Complex adjoint of a quaternion matrix X = X1 + X2 j: [[X1, X2], [-conj X2, conj X1]].

    Textbook injective ring homomorphism: chi(XY) = chi(X) chi(Y).
    """
    X1 = X[0] + 1j * X[1]
    X2 = X[2] + 1j * X[3]
    top = np.concatenate([X1, X2], axis=-1)
    bot = np.concatenate([-np.conj(X2), np.conj(X1)], axis=-1)
    return np.concatenate([top, bot], axis=-2)


def chi_inv(M):
    m = M.shape[-2] // 2
    n = M.shape[-1] // 2
    X1 = M[..., :m, :n]
    X2 = M[..., :m, n:]
    return np.stack([X1.real, X1.imag, X2.real, X2.imag])


# ---------------------------------------------------------------- scalars


def test_unit_table_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "quaternion_units.json")))
    for x, row in g["products"].items():
        for y, (sign, unit) in row.items():
            ex = np.zeros(4)
            ey = np.zeros(4)
            ex[UNITS[x]] = 1.0
            ey[UNITS[y]] = 1.0
            want = np.zeros(4)
            want[UNITS[unit]] = sign
            np.testing.assert_array_equal(Q.hamilton(ex, ey), want, err_msg=f"{x}*{y}")


def test_hamilton_is_complex_adjoint_homomorphism():
    rng = np.random.default_rng(10)
    x = rand_q(rng, 50)
    y = rand_q(rng, 50)
    xy = Q.hamilton(x, y)
    for e in range(50):
        lhs = chi(xy[:, e].reshape(4, 1, 1))
        rhs = chi(x[:, e].reshape(4, 1, 1)) @ chi(y[:, e].reshape(4, 1, 1))
        np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_hamilton_norm_is_multiplicative_and_noncommutative():
    rng = np.random.default_rng(11)
    x = rand_q(rng, 100)
    y = rand_q(rng, 100)
    nx = np.sqrt((x * x).sum(0))
    ny = np.sqrt((y * y).sum(0))
    nxy = np.sqrt((Q.hamilton(x, y) ** 2).sum(0))
    np.testing.assert_allclose(nxy, nx * ny, rtol=1e-13)
    assert np.abs(Q.hamilton(x, y) - Q.hamilton(y, x)).max() > 1e-3


def test_qmatmul_matches_complex_adjoint():
    rng = np.random.default_rng(12)
    X = rand_q(rng, 5, 7)
    Y = rand_q(rng, 7, 3)
    np.testing.assert_allclose(chi(Q.qmatmul(X, Y)), chi(X) @ chi(Y), atol=1e-12)


# ---------------------------------------------------------------- definition


def tprod_python_loops(A, B):
    """Brute force over every (i, t, k, r, j) with scalar products through chi."""
    _, m, n, p = A.shape
    s = B.shape[2]
    C = np.zeros((4, m, s, p))
    for i in range(m):
        for t in range(s):
            for k in range(p):
                acc = np.zeros((2, 2), dtype=complex)
                for r in range(p):
                    for j in range(n):
                        acc = acc + chi(A[:, i, j, r].reshape(4, 1, 1)) @ chi(
                            B[:, j, t, (k - r) % p].reshape(4, 1, 1))
                C[:, i, t, k] = chi_inv(acc)[:, 0, 0]
    return C


@pytest.mark.parametrize("m,n,s,p", [(2, 3, 2, 1), (3, 2, 2, 2), (2, 2, 3, 3), (1, 3, 2, 4)])
def test_definition_matches_python_loops(m, n, s, p):
    rng = np.random.default_rng(100 + p)
    A = rand_q(rng, m, n, p)
    B = rand_q(rng, n, s, p)
    np.testing.assert_allclose(Q.tprod_def(A, B), tprod_python_loops(A, B), atol=1e-12)


@pytest.mark.parametrize("m,n,s,p", [(3, 4, 5, 1), (4, 3, 2, 2), (5, 4, 3, 3), (3, 5, 4, 7), (8, 8, 8, 16)])
def test_definition_matches_explicit_bcirc(m, n, s, p):
    rng = np.random.default_rng(200 + p)
    A = rand_q(rng, m, n, p)
    B = rand_q(rng, n, s, p)
    np.testing.assert_allclose(Q.tprod_def(A, B), Q.tprod_bcirc(A, B), atol=1e-12)


def test_bcirc_layout_matches_paper():
    # First block column is A^(1..p), first block row is A^(1), A^(p), ..., A^(2) (eq. bcirc-unfold).
    p = 4
    A = np.zeros((4, 1, 1, p))
    A[0, 0, 0, :] = [1, 2, 3, 4]
    M = Q.bcirc(A)[0]
    np.testing.assert_array_equal(M[:, 0], [1, 2, 3, 4])
    np.testing.assert_array_equal(M[0, :], [1, 4, 3, 2])


def test_p1_is_quaternion_matrix_product_A_left():
    rng = np.random.default_rng(13)
    A = rand_q(rng, 4, 6, 1)
    B = rand_q(rng, 6, 5, 1)
    C = Q.tprod_def(A, B)[..., 0]
    want = chi_inv(chi(A[..., 0]) @ chi(B[..., 0]))
    np.testing.assert_allclose(C, want, atol=1e-12)
    wrong = chi_inv(chi(np.swapaxes(B[..., 0], 1, 2)) @ chi(np.swapaxes(A[..., 0], 1, 2)))
    assert np.abs(C - np.swapaxes(wrong, 1, 2)).max() > 1e-3


@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_real_case_is_real_tproduct_via_fft(p):
    # Alg. 2.1 for real tensors: C_hat(:,:,r) = A_hat(:,:,r) B_hat(:,:,r) with numpy's FFT.
    rng = np.random.default_rng(14 + p)
    A = np.zeros((4, 4, 3, p))
    B = np.zeros((4, 3, 5, p))
    A[0] = rng.standard_normal((4, 3, p))
    B[0] = rng.standard_normal((3, 5, p))
    Ah = np.fft.fft(A[0], axis=-1)
    Bh = np.fft.fft(B[0], axis=-1)
    Ch = np.einsum("mnp,nsp->msp", Ah, Bh)
    want = np.fft.ifft(Ch, axis=-1)
    C = Q.tprod_def(A, B)
    np.testing.assert_allclose(C[0], want.real, atol=1e-12)
    np.testing.assert_allclose(C[1:], 0.0, atol=0)


@pytest.mark.parametrize("p", [3, 6])
def test_complex_case_is_complex_tproduct_via_fft(p):
    rng = np.random.default_rng(15 + p)
    A = np.zeros((4, 3, 4, p))
    B = np.zeros((4, 4, 2, p))
    A[:2] = rng.standard_normal((2, 3, 4, p))
    B[:2] = rng.standard_normal((2, 4, 2, p))
    Ah = np.fft.fft(A[0] + 1j * A[1], axis=-1)
    Bh = np.fft.fft(B[0] + 1j * B[1], axis=-1)
    want = np.fft.ifft(np.einsum("mnp,nsp->msp", Ah, Bh), axis=-1)
    C = Q.tprod_def(A, B)
    np.testing.assert_allclose(C[0] + 1j * C[1], want, atol=1e-12)
    np.testing.assert_allclose(C[2:], 0.0, atol=0)


def test_identity_tensor():
    rng = np.random.default_rng(16)
    A = rand_q(rng, 4, 5, 6)
    np.testing.assert_allclose(Q.tprod_def(A, Q.identity(5, 6)), A, atol=1e-14)
    np.testing.assert_allclose(Q.tprod_def(Q.identity(4, 6), A), A, atol=1e-14)


def test_associativity():
    rng = np.random.default_rng(17)
    A = rand_q(rng, 3, 4, 5)
    B = rand_q(rng, 4, 2, 5)
    D = rand_q(rng, 2, 3, 5)
    lhs = Q.tprod_def(Q.tprod_def(A, B), D)
    rhs = Q.tprod_def(A, Q.tprod_def(B, D))
    assert Q.rel_fro(lhs, rhs) < 1e-14


def test_bcirc_is_multiplicative():
    # bcirc(A*B) = bcirc(A) bcirc(B), used in the proof of Thm 5.1.
    rng = np.random.default_rng(18)
    A = rand_q(rng, 3, 4, 5)
    B = rand_q(rng, 4, 2, 5)
    lhs = Q.bcirc(Q.tprod_def(A, B))
    rhs = Q.qmatmul(Q.bcirc(A), Q.bcirc(B))
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_conj_transpose_rules():
    rng = np.random.default_rng(19)
    X = rand_q(rng, 3, 4, 5)
    np.testing.assert_allclose(Q.bcirc(Q.conj_transpose(X)), Q.qmat_conj_transpose(Q.bcirc(X)), atol=0)
    A = rand_q(rng, 3, 4, 6)
    B = rand_q(rng, 4, 2, 6)
    lhs = Q.conj_transpose(Q.tprod_def(A, B))
    rhs = Q.tprod_def(Q.conj_transpose(B), Q.conj_transpose(A))
    assert Q.rel_fro(lhs, rhs) < 1e-14


def test_columns_and_entries_match_full_definition():
    rng = np.random.default_rng(20)
    A = rand_q(rng, 5, 6, 7)
    B = rand_q(rng, 6, 8, 7)
    C = Q.tprod_def(A, B)
    ts = [0, 3, 7]
    np.testing.assert_allclose(Q.tprod_def_columns(A, B, ts), C[:, :, ts, :], atol=1e-12)
    ii, tt, kk = rng.integers(0, 5, 30), rng.integers(0, 8, 30), rng.integers(0, 7, 30)
    np.testing.assert_allclose(Q.tprod_def_entries(A, B, ii, tt, kk), C[:, ii, tt, kk], atol=1e-12)
    np.testing.assert_allclose(Q.tprod_def_pairs(A, B, tt, kk), C[:, :, tt, kk], atol=1e-12)


# ---------------------------------------------------------------- Alg. 5.1 and Example 3.1


@pytest.mark.parametrize("m,n,s,p", [(3, 4, 5, 1), (3, 4, 5, 2), (4, 3, 2, 3), (5, 4, 3, 7),
                                     (6, 5, 4, 12), (4, 4, 4, 31), (3, 2, 3, 100)])
def test_alg51_matches_definition(m, n, s, p):
    rng = np.random.default_rng(300 + p)
    A = rand_q(rng, m, n, p)
    B = rand_q(rng, n, s, p)
    assert Q.rel_fro(Q.alg51(A, B), Q.tprod_def(A, B)) < 1e-14


def test_alg51_reproduces_table1_error_level():
    rows = json.load(open(os.path.join(GOLDEN, "table1_errors.json")))["rows"]
    rng = np.random.default_rng(21)
    checked = 0
    for r in rows:
        if r["m"] * r["n"] * r["s"] * r["p"] ** 2 > 100 * 100 * 100 * 10 ** 2:
            continue  # definition too slow for the CPU suite
        A = rand_q(rng, r["m"], r["n"], r["p"])
        B = rand_q(rng, r["n"], r["s"], r["p"])
        err = Q.rel_fro(Q.alg51(A, B), Q.tprod_def(A, B))
        assert err < 2e-15, (r, err)
        checked += 1
    assert checked >= 2


def test_naive_port_fails_for_p_ge_3():
    rng = np.random.default_rng(22)
    for p in (3, 4, 8):
        A = rand_q(rng, 4, 5, p)
        B = rand_q(rng, 5, 3, p)
        assert Q.rel_fro(Q.naive_alg21(A, B), Q.tprod_def(A, B)) > 0.1
    for p in (1, 2):
        A = rand_q(rng, 4, 5, p)
        B = rand_q(rng, 5, 3, p)
        assert Q.rel_fro(Q.naive_alg21(A, B), Q.tprod_def(A, B)) < 1e-14
    A = rand_q(rng, 4, 5, 6)
    B = rand_q(rng, 5, 3, 6)
    A[2:] = 0
    B[2:] = 0
    assert Q.rel_fro(Q.naive_alg21(A, B), Q.tprod_def(A, B)) < 1e-14


def _dft(p, normalised):
    w = np.exp(-2j * np.pi / p)
    F = np.array([[w ** (r * c) for c in range(p)] for r in range(p)])
    return F / np.sqrt(p) if normalised else F


def _cplx_as_quat(M):
    return np.stack([M.real, M.imag, np.zeros_like(M.real), np.zeros_like(M.real)])


def test_eq_F4_example_pattern():
    g = json.load(open(os.path.join(GOLDEN, "eq_F4.json")))
    gen = g["A_generators_j_coefficient"]
    p = len(gen)
    A = np.zeros((4, p, p))
    for r in range(p):
        for c in range(p):
            A[2, r, c] = gen[(r - c) % p]       # circ(j, 2j, 3j, 4j), eq. circulant
    for normalised, scale in ((False, 1.0), (True, 0.25)):
        F = _dft(p, normalised)
        R = Q.qmatmul(Q.qmatmul(_cplx_as_quat(F), A), _cplx_as_quat(F.conj().T))
        mag = np.sqrt((R ** 2).sum(0))
        want = np.zeros((p, p))
        for key, v in g["expected_magnitudes_unnormalised"].items():
            i, j = (int(t) - 1 for t in key.split(","))
            want[i, j] = v * scale
        np.testing.assert_allclose(mag, want, atol=1e-12)
        assert np.abs(R[0:2]).max() < 1e-12          # no 1, i parts: the print dropped a j
        assert mag[1, 3] > 1.0                       # off-diagonal: F_4 does not diagonalise


def test_example31_split_identity():
    # F A F^* = F A1 F^* + (F A2 F) j for a circulant quaternion A (Example 3.1).
    rng = np.random.default_rng(23)
    p = 6
    gen = rng.standard_normal((4, p))
    A = np.zeros((4, p, p))
    for r in range(p):
        for c in range(p):
            A[:, r, c] = gen[:, (r - c) % p]
    F = _dft(p, True)
    lhs = Q.qmatmul(Q.qmatmul(_cplx_as_quat(F), A), _cplx_as_quat(F.conj().T))
    A1 = A[0] + 1j * A[1]
    A2 = A[2] + 1j * A[3]
    part1 = F @ A1 @ F.conj().T
    part2 = F @ A2 @ F
    want = np.stack([part1.real, part1.imag, part2.real, part2.imag])
    np.testing.assert_allclose(lhs, want, atol=1e-12)
    # the first part is diagonal, the second is not in general
    assert np.abs(part1 - np.diag(np.diag(part1))).max() < 1e-12
    assert np.abs(part2 - np.diag(np.diag(part2))).max() > 1e-3


# ---------------------------------------------------------------- gradient


def test_gradient_central_differences():
    rng = np.random.default_rng(24)
    A = rand_q(rng, 3, 4, 5)
    B = rand_q(rng, 4, 3, 5)
    T = rand_q(rng, 3, 3, 5)
    dA, dB = Q.grad_def(A, B, T)
    h = 1e-3
    for X, dX in ((A, dA), (B, dB)):
        for _ in range(12):
            idx = tuple(int(rng.integers(0, d)) for d in X.shape)
            Xp = X.copy()
            Xm = X.copy()
            Xp[idx] += h
            Xm[idx] -= h
            if X is A:
                fd = (Q.loss_def(Xp, B, T) - Q.loss_def(Xm, B, T)) / (2 * h)
            else:
                fd = (Q.loss_def(A, Xp, T) - Q.loss_def(A, Xm, T)) / (2 * h)
            assert abs(fd - dX[idx]) <= 1e-7 * max(1.0, abs(fd)), (idx, fd, dX[idx])
    for _ in range(4):
        VA = rand_q(rng, *A.shape[1:])
        VB = rand_q(rng, *B.shape[1:])
        fd = (Q.loss_def(A + h * VA, B + h * VB, T) - Q.loss_def(A - h * VA, B - h * VB, T)) / (2 * h)
        an = float(np.sum(dA * VA) + np.sum(dB * VB))
        # loss is quartic along a joint direction: central difference error is O(h^2)
        assert abs(fd - an) <= 1e-4 * max(1.0, abs(an))


# ---------------------------------------------------------------- planted mistakes


def _unit_table_ok(hfun):
    g = json.load(open(os.path.join(GOLDEN, "quaternion_units.json")))
    for x, row in g["products"].items():
        for y, (sign, unit) in row.items():
            ex = np.zeros(4)
            ey = np.zeros(4)
            ex[UNITS[x]] = 1.0
            ey[UNITS[y]] = 1.0
            want = np.zeros(4)
            want[UNITS[unit]] = sign
            if not np.array_equal(hfun(ex, ey), want):
                return False
    return True


def test_pins_catch_planted_mistakes(monkeypatch):
    """Each plausible slip in the oracle is caught by at least one pin above."""
    rng = np.random.default_rng(25)
    A = rand_q(rng, 2, 3, 3)
    B = rand_q(rng, 3, 2, 3)
    ref_loops = tprod_python_loops(A, B)

    # (1) a sign error in one Hamilton term
    good = Q.hamilton

    def bad_hamilton(x, y):
        r = good(x, y)
        a1, b1, c1, d1 = x
        a2, b2, c2, d2 = y
        r[3] = a1 * d2 + b1 * c2 + c1 * b2 + d1 * a2
        return r
    assert _unit_table_ok(good)
    assert not _unit_table_ok(bad_hamilton)

    # (2) a wrong circulant index (k + r instead of k - r)
    def bad_def(A, B):
        p = A.shape[-1]
        C = np.zeros((4, A.shape[1], B.shape[2], p))
        for k in range(p):
            for r in range(p):
                C[..., k] += Q.qmatmul(A[..., r], B[..., (k + r) % p])
        return C
    assert np.abs(bad_def(A, B) - ref_loops).max() > 1e-3

    # (3) transposed operand order B . A
    def bad_order(A, B):
        p = A.shape[-1]
        C = np.zeros((4, A.shape[1], B.shape[2], p))
        for k in range(p):
            for r in range(p):
                X = np.swapaxes(B[..., (k - r) % p], 1, 2)
                Y = np.swapaxes(A[..., r], 1, 2)
                C[..., k] += np.swapaxes(Q.qmatmul(X, Y), 1, 2)
        return C
    assert np.abs(bad_order(A, B) - ref_loops).max() > 1e-3

    # (4) Alg. 5.1 without the frequency reversal fails the definition check
    def bad_alg51(A, B):
        A1, A2 = Q.cd_split(A)
        B1, B2 = Q.cd_split(B)
        Ah1, Ah2 = np.fft.fft(np.conj(A1), axis=-1), -np.fft.fft(A2, axis=-1)
        Bh1, Bh2 = np.fft.fft(np.conj(B1), axis=-1), -np.fft.fft(B2, axis=-1)
        Ch1 = np.einsum("mnp,nsp->msp", Ah1, Bh1) - np.einsum("mnp,nsp->msp", np.conj(Ah2), Bh2)
        Ch2 = np.einsum("mnp,nsp->msp", np.conj(Ah1), Bh2) + np.einsum("mnp,nsp->msp", Ah2, Bh1)
        return Q.cd_join(np.fft.ifft(np.conj(Ch1), axis=-1), -np.fft.ifft(Ch2, axis=-1))
    assert Q.rel_fro(bad_alg51(A, B), ref_loops) > 1e-3
