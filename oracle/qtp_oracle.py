"""FP64 CPU oracle for the T-product of third-order quaternion tensors.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA path.

Representation
--------------
A quaternion tensor X in Q^{m x n x p} is a float64 ndarray of shape
``(4, m, n, p)`` holding the real components (a, b, c, d) of
q = a + b i + c j + d k  (paper, Sec. 1).  A quaternion matrix is ``(4, m, n)``.

What is computed
----------------
* ``hamilton``            Hamilton product of quaternions (Sec. 1 rules
                          i^2 = j^2 = k^2 = ijk = -1).
* ``qmatmul``             quaternion matrix product, A on the left.
* ``bcirc/unfold/fold``   the operators of Sec. 2.4, eq. (bcirc-unfold).
* ``tprod_bcirc``         Definition 2.3 literally: fold(bcirc(A) . unfold(B)).
* ``tprod_def``           the same definition as a sum over frontal slices,
                          C^(k) = sum_r A^(r) B^((k - r) mod p) (0-based), which
                          is row block k of bcirc(A) times unfold(B).
* ``tprod_def_columns``   lateral columns C(:, t, :) by the definition.
* ``tprod_def_pairs``     mode-1 fibres C(:, t, k) by the definition.
* ``tprod_def_entries``   single entries C(i, t, k) by the definition.
* ``alg51``               Algorithm 5.1 in FP64 (Thm 5.1, eqs. TC/TC2, ifft-C),
                          used only for the self-tests and as a CPU timing.
* ``naive_alg21``         Algorithm 2.1 applied blindly to quaternion slices
                          (F_p on both Cayley-Dickson halves); wrong for p >= 3
                          (Example 3.1) - kept as a negative control.
* ``conj_transpose``,     tensor conjugate transpose and identity tensor
  ``identity``            (Kilmer-Martin convention; the paper defines none).
* ``grad_def``            gradient of ||A*B - T||_F^2 by the definition.

Parity pins: every function above is checked in ``tests/test_oracle_pins.py``
against values the paper prints or that mathematics fixes (unit table, the
complex-adjoint homomorphism, FFT-based real/complex T-products, explicit
bcirc brute force, identity/associativity/adjoint invariants, Table 1's error
level, Example 3.1 / eq. F4, central finite differences).  No function here is
"parity unpinned".
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------
# Scalars and matrices (Sec. 1, Sec. 2.2)
# --------------------------------------------------------------------------


def hamilton(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Hamilton product x*y of quaternion arrays with leading axis 4.

    Follows the multiplication rules of Sec. 1: i^2 = j^2 = k^2 = ijk = -1,
    ij = -ji = k, jk = -kj = i, ki = -ik = j.
    """
    a1, b1, c1, d1 = x
    a2, b2, c2, d2 = y
    return np.stack([
        a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2,
        a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2,
        a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2,
        a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2,
    ])


def qconj(x: np.ndarray) -> np.ndarray:
    """Quaternion conjugate a - b i - c j - d k, component-wise."""
    return np.stack([x[0], -x[1], -x[2], -x[3]])


def qmatmul(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Quaternion matrix product X . Y, X (4, m, n) on the left of Y (4, n, s).

    Entry (i, t) is sum_j X_ij * Y_jt with * the Hamilton product; the sum over
    j is done by real matrix products (a library primitive), one per pair of
    components, with the signs of ``hamilton``.  Leading batch axes between the
    component axis and the last two axes broadcast.
    """
    a1, b1, c1, d1 = X
    a2, b2, c2, d2 = Y
    mm = np.matmul
    return np.stack([
        mm(a1, a2) - mm(b1, b2) - mm(c1, c2) - mm(d1, d2),
        mm(a1, b2) + mm(b1, a2) + mm(c1, d2) - mm(d1, c2),
        mm(a1, c2) - mm(b1, d2) + mm(c1, a2) + mm(d1, b2),
        mm(a1, d2) + mm(b1, c2) - mm(c1, b2) + mm(d1, a2),
    ])


def qmat_conj_transpose(X: np.ndarray) -> np.ndarray:
    """Conjugate transpose X^* of a quaternion matrix (4, m, n) -> (4, n, m)."""
    return np.swapaxes(qconj(X), -1, -2)


# --------------------------------------------------------------------------
# Tensor operators (Sec. 2.4, eq. bcirc-unfold)
# --------------------------------------------------------------------------


def bcirc(A: np.ndarray) -> np.ndarray:
    """Block circulant matrix (4, m p, n p) of A (4, m, n, p).

    Block (r, c) (0-based) is the frontal slice A^((r - c) mod p): the first
    block column is A^(1), ..., A^(p) and each block column is the previous one
    shifted down by one block (eq. bcirc-unfold).
    """
    _, m, n, p = A.shape
    out = np.zeros((4, m * p, n * p))
    for r in range(p):
        for c in range(p):
            out[:, r * m:(r + 1) * m, c * n:(c + 1) * n] = A[:, :, :, (r - c) % p]
    return out


def unfold(B: np.ndarray) -> np.ndarray:
    """Stack the frontal slices of B (4, n, s, p) into a (4, n p, s) block column."""
    _, n, s, p = B.shape
    return np.concatenate([B[:, :, :, k] for k in range(p)], axis=1)


def fold(X: np.ndarray, p: int) -> np.ndarray:
    """Inverse of ``unfold``: (4, m p, s) -> (4, m, s, p)."""
    _, mp, s = X.shape
    m = mp // p
    return np.stack([X[:, k * m:(k + 1) * m, :] for k in range(p)], axis=-1)


def tprod_bcirc(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Definition 2.3 taken literally: fold(bcirc(A) . unfold(B))."""
    p = A.shape[-1]
    assert B.shape[-1] == p and A.shape[2] == B.shape[1]
    return fold(qmatmul(bcirc(A), unfold(B)), p)


def tprod_def(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """T-product by its definition, slice by slice.

    Row block k of bcirc(A) is (A^(k), A^(k-1), ..., A^(k-p+1)) (indices mod
    p), so frontal slice k of fold(bcirc(A) unfold(B)) is
    C^(k) = sum_r A^(r) . B^((k - r) mod p), A on the left (Def. 2.3).
    Cost 16 m n s p^2 real multiplications (Thm 5.2).
    """
    _, m, n, p = A.shape
    _, n2, s, p2 = B.shape
    assert n == n2 and p == p2
    C = np.zeros((4, m, s, p))
    for k in range(p):
        acc = np.zeros((4, m, s))
        for r in range(p):
            acc += qmatmul(A[:, :, :, r], B[:, :, :, (k - r) % p])
        C[:, :, :, k] = acc
    return C


def tprod_def_columns(A: np.ndarray, B: np.ndarray, ts) -> np.ndarray:
    """Lateral columns C(:, t, :) for t in ``ts`` by the definition.

    Uses Def. 2.3 restricted to the chosen columns of B: slice k of the result
    is row block k of bcirc(A), i.e. the (m, n p) quaternion matrix
    [A^(k), A^(k-1), ..., A^(k-p+1)], times unfold(B(:, ts, :)).
    Returns (4, m, len(ts), p).
    """
    _, m, n, p = A.shape
    ts = np.asarray(ts)
    Bt = B[:, :, ts, :]                                   # (4, n, T, p)
    # unfold(B(:, ts, :)) with slice r at rows r n .. r n + n - 1
    UB = np.concatenate([Bt[:, :, :, r] for r in range(p)], axis=1)   # (4, n p, T)
    C = np.zeros((4, m, len(ts), p))
    for k in range(p):
        row_block = np.concatenate([A[:, :, :, (k - c) % p] for c in range(p)], axis=2)
        C[:, :, :, k] = qmatmul(row_block, UB)
    return C


def tprod_def_pairs(A: np.ndarray, B: np.ndarray, tt, kk) -> np.ndarray:
    """Mode-1 fibres C(:, t, k) for the pairs (t, k) in zip(tt, kk), by the definition.

    C(i, t, k) = sum_r sum_j A(i, j, r) * B(j, t, (k - r) mod p): row i of row
    block k of bcirc(A) times column t of unfold(B) (Def. 2.3).  All pairs go
    through one quaternion matrix product: A as the (m, n p) matrix over (j, r)
    times the (n p, P) matrix whose column q holds B(j, t_q, (k_q - r) mod p).
    Returns (4, m, P).
    """
    _, m, n, p = A.shape
    tt, kk = np.asarray(tt), np.asarray(kk)
    r = np.arange(p)
    cols = np.empty((4, n, p, len(tt)))
    for q in range(len(tt)):
        cols[:, :, :, q] = B[:, :, tt[q], :][:, :, (kk[q] - r) % p]
    return qmatmul(A.reshape(4, m, n * p), cols.reshape(4, n * p, len(tt)))


def tprod_def_entries(A: np.ndarray, B: np.ndarray, ii, tt, kk) -> np.ndarray:
    """Single entries C(i, t, k) = sum_r sum_j A(i, j, r) * B(j, t, (k - r) mod p).

    The sum runs over the n p products of row i of row block k of bcirc(A)
    with column t of unfold(B) (Def. 2.3).  Returns (4, len(ii)).
    """
    _, m, n, p = A.shape
    ii, tt, kk = (np.asarray(v) for v in (ii, tt, kk))
    out = np.zeros((4, len(ii)))
    r = np.arange(p)
    for e in range(len(ii)):
        arow = A[:, ii[e], :, :]                          # (4, n, p) over (j, r)
        bcol = B[:, :, tt[e], :][:, :, (kk[e] - r) % p]   # (4, n, p) over (j, r)
        out[:, e] = hamilton(arow, bcol).sum(axis=(1, 2))
    return out


# --------------------------------------------------------------------------
# Conventions the paper does not define (Kilmer-Martin)
# --------------------------------------------------------------------------


def conj_transpose(X: np.ndarray) -> np.ndarray:
    """Tensor conjugate transpose: X^H(:,:,1) = X(:,:,1)^*, X^H(:,:,k) = X(:,:,p+2-k)^*.

    0-based: slice k of X^H is the quaternion conjugate transpose of slice
    (-k) mod p of X, which makes bcirc(X^H) = bcirc(X)^*.
    """
    p = X.shape[-1]
    return np.stack([qmat_conj_transpose(X[:, :, :, (-k) % p]) for k in range(p)], axis=-1)


def identity(n: int, p: int) -> np.ndarray:
    """Identity tensor: first frontal slice I_n (real), the others zero."""
    out = np.zeros((4, n, n, p))
    out[0, :, :, 0] = np.eye(n)
    return out


# --------------------------------------------------------------------------
# Algorithm 5.1 (Sec. 5) and the negative control (Alg. 2.1, Example 3.1)
# --------------------------------------------------------------------------


def cd_split(X: np.ndarray):
    """Cayley-Dickson halves X = X1 + X2 j with X1 = a + b i, X2 = c + d i (Sec. 2.2)."""
    return X[0] + 1j * X[1], X[2] + 1j * X[3]


def cd_join(X1: np.ndarray, X2: np.ndarray) -> np.ndarray:
    """Quaternion components (a, b, c, d) of X1 + X2 j."""
    return np.stack([X1.real, X1.imag, X2.real, X2.imag])


def alg51(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Algorithm 5.1 in FP64.

    Step 1 (eq. fftA-B, eq. fft-Q): A_hat = fft(conj(A1)) - fft(A2) j along
    mode 3, i.e. A_hat_1 = fft(conj A1), A_hat_2 = -fft(A2); the same for B.
    ``fft`` is unnormalised with omega = exp(-2 pi i / p) (eq. DFT, Prop. 2.1).
    Step 2 (eqs. TC, TC2) with the 1-based index p+2-i written 0-based as
    g = (-f) mod p (the wrap A_hat(:,:,p+1) := A_hat(:,:,1) is the g = 0 case):
      C_hat_1(f) = A_hat_1(g) B_hat_1(g) - conj(A_hat_2(f)) B_hat_2(g)
      C_hat_2(f) = conj(A_hat_1(g)) B_hat_2(f) + A_hat_2(f) B_hat_1(f)
    Step 3 (eq. ifft-C): C = ifft(conj C_hat_1) - ifft(C_hat_2) j.
    """
    p = A.shape[-1]
    A1, A2 = cd_split(A)
    B1, B2 = cd_split(B)
    Ah1 = np.fft.fft(np.conj(A1), axis=-1)
    Ah2 = -np.fft.fft(A2, axis=-1)
    Bh1 = np.fft.fft(np.conj(B1), axis=-1)
    Bh2 = -np.fft.fft(B2, axis=-1)
    m, s = A.shape[1], B.shape[2]
    Ch1 = np.zeros((m, s, p), dtype=complex)
    Ch2 = np.zeros((m, s, p), dtype=complex)
    for f in range(p):
        g = (-f) % p
        Ch1[:, :, f] = Ah1[:, :, g] @ Bh1[:, :, g] - np.conj(Ah2[:, :, f]) @ Bh2[:, :, g]
        Ch2[:, :, f] = np.conj(Ah1[:, :, g]) @ Bh2[:, :, f] + Ah2[:, :, f] @ Bh1[:, :, f]
    C1 = np.fft.ifft(np.conj(Ch1), axis=-1)
    C2 = -np.fft.ifft(Ch2, axis=-1)
    return cd_join(C1, C2)


def naive_alg21(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Algorithm 2.1 applied to quaternion tensors without the octonion correction.

    F_p is applied to both Cayley-Dickson halves (A_hat_r = fft(A_r)), each
    frequency slice is multiplied as a quaternion matrix in CD form,
    (P1 + P2 j)(Q1 + Q2 j) = (P1 Q1 - P2 conj(Q2)) + (P1 Q2 + P2 conj(Q1)) j,
    and the halves are inverse transformed.  Example 3.1 shows why this is not
    the T-product in general: j c = conj(c) j turns F_p into conj(F_p) on the j
    half.  Kept only as the negative control.
    """
    A1, A2 = cd_split(A)
    B1, B2 = cd_split(B)
    Ah1, Ah2 = np.fft.fft(A1, axis=-1), np.fft.fft(A2, axis=-1)
    Bh1, Bh2 = np.fft.fft(B1, axis=-1), np.fft.fft(B2, axis=-1)
    Ch1 = np.einsum('mnp,nsp->msp', Ah1, Bh1) - np.einsum('mnp,nsp->msp', Ah2, np.conj(Bh2))
    Ch2 = np.einsum('mnp,nsp->msp', Ah1, Bh2) + np.einsum('mnp,nsp->msp', Ah2, np.conj(Bh1))
    return cd_join(np.fft.ifft(Ch1, axis=-1), np.fft.ifft(Ch2, axis=-1))


# --------------------------------------------------------------------------
# Loss and gradient (training-style use of the product; not in the paper)
# --------------------------------------------------------------------------


def loss_def(A: np.ndarray, B: np.ndarray, T: np.ndarray) -> float:
    """||A*B - T||_F^2 over all four real components, A*B by the definition."""
    R = tprod_def(A, B) - T
    return float(np.sum(R * R))


def grad_def(A: np.ndarray, B: np.ndarray, T: np.ndarray):
    """Gradient of ||A*B - T||_F^2 with each quaternion entry as four reals.

    dC = 2 (C - T), dA = dC * B^H, dB = A^H * dC, every product by the
    definition.  This follows from Re tr(XY) = Re tr(YX) for quaternion
    matrices and bcirc(X^H) = bcirc(X)^*.
    """
    dC = 2.0 * (tprod_def(A, B) - T)
    dA = tprod_def(dC, conj_transpose(B))
    dB = tprod_def(conj_transpose(A), dC)
    return dA, dB


# --------------------------------------------------------------------------
# Error metric (Table 1 "error"; the paper states no norm)
# --------------------------------------------------------------------------


def rel_fro(x: np.ndarray, ref: np.ndarray) -> float:
    """||x - ref||_F / ||ref||_F over all real components."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.sqrt(np.sum(ref * ref))
    num = np.sqrt(np.sum((x - ref) ** 2))
    return float(num / den) if den > 0 else float(num)
