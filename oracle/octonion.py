"""FP64 octonion algebra of Sec. 2.2 and Sec. 4, and the octonion-domain route
to the T-product of Theorem 5.1.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this module: only ``tests/`` use it.  It shares no code with the CUDA path and
none with ``oracle.alg51`` (no FFT here: every transform is an octonion matrix
product with the DFT matrix of eq. DFT).

Representation
--------------
An octonion o = a + b i + c j + d k + e l + f il + g jl + h kl (Sec. 2.2) is a
float64 array with leading axis 8 in that basis order; an octonion matrix is
``(8, rows, cols)``.  A quaternion array ``(4, ...)`` (the layout of
``oracle.qtp_oracle``) embeds as the first four components.

Reading of the products
-----------------------
The paper writes products of three or more octonions without brackets
(Prop. 4.1 (ii)-(v), eq. relation-remark, Prop. 4.2, Thm 4.2, Thm 5.1).  Every
such product is read left to right, ((x y) z) ...; brackets the paper writes
are kept.  For matrices this is the entry-wise reading ((X Y) Z)_ij =
sum_kl (X_ik Y_kl) Z_lj.  A complex number times a unit, ``p l`` or
``p (jl)``, is the octonion product of the complex number p = a + b i (as an
octonion) with the unit.

Parity pins (``tests/test_oracle_octonion.py``): the product against the
paper's multiplication table (golden fixture) and against a Cayley-Dickson
doubling of the Hamilton product, the composition law |x y| = |x| |y|,
alternativity and the Moufang identity; every proposition and theorem of
Sec. 4 used here is then checked numerically, and ``tprod_octonion`` against
the T-product definition.  No function here is "parity unpinned".
"""
from __future__ import annotations

import numpy as np

BASIS = ("1", "i", "j", "k", "l", "il", "jl", "kl")


# --------------------------------------------------------------------------
# Scalars (Sec. 2.2)
# --------------------------------------------------------------------------


def omul(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Octonion product x y, component by component as Sec. 2.2 writes it out
    from the multiplication table (leading axis 8, broadcasting the rest)."""
    a1, b1, c1, d1, e1, f1, g1, h1 = x
    a2, b2, c2, d2, e2, f2, g2, h2 = y
    return np.stack([
        a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2 - e1 * e2 - f1 * f2 - g1 * g2 - h1 * h2,
        a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2 + e1 * f2 - f1 * e2 + h1 * g2 - g1 * h2,
        a1 * c2 + c1 * a2 + d1 * b2 - b1 * d2 + e1 * g2 - g1 * e2 + f1 * h2 - h1 * f2,
        a1 * d2 + d1 * a2 + b1 * c2 - c1 * b2 + e1 * h2 - h1 * e2 + g1 * f2 - f1 * g2,
        a1 * e2 + e1 * a2 + f1 * b2 - b1 * f2 + g1 * c2 - c1 * g2 + h1 * d2 - d1 * h2,
        a1 * f2 + f1 * a2 + b1 * e2 - e1 * b2 + h1 * c2 - c1 * h2 + d1 * g2 - g1 * d2,
        a1 * g2 + g1 * a2 + b1 * h2 - h1 * b2 + c1 * e2 - e1 * c2 + f1 * d2 - d1 * f2,
        a1 * h2 + h1 * a2 + g1 * b2 - b1 * g2 + c1 * f2 - f1 * c2 + d1 * e2 - e1 * d2,
    ])


def oconj(x: np.ndarray) -> np.ndarray:
    """Conjugate a - b i - ... - h kl (eq. conj)."""
    out = -np.asarray(x, dtype=np.float64).copy()
    out[0] = -out[0]
    return out


def onorm(x: np.ndarray) -> np.ndarray:
    """Modulus |o| = sqrt(conj(o) o) = the Euclidean norm of the 8 components."""
    return np.sqrt(np.sum(np.asarray(x) ** 2, axis=0))


def unit(name: str) -> np.ndarray:
    """The basis octonion ``name`` (one of BASIS)."""
    out = np.zeros(8)
    out[BASIS.index(name)] = 1.0
    return out


def from_complex(z) -> np.ndarray:
    """Complex z = a + b i (any shape) as octonions (8, ...)."""
    z = np.asarray(z, dtype=complex)
    out = np.zeros((8,) + z.shape)
    out[0], out[1] = z.real, z.imag
    return out


def from_quat(q: np.ndarray) -> np.ndarray:
    """Quaternion components (4, ...) as octonions (8, ...) with zero l part."""
    q = np.asarray(q, dtype=np.float64)
    return np.concatenate([q, np.zeros_like(q)], axis=0)


def to_quat(o: np.ndarray, tol: float = 1e-9) -> np.ndarray:
    """The quaternion part (4, ...) of octonions whose l part is zero; raises
    if the l part exceeds ``tol`` times the largest component."""
    o = np.asarray(o)
    scale = max(float(np.max(np.abs(o))), 1.0)
    if np.max(np.abs(o[4:]), initial=0.0) > tol * scale:
        raise ValueError("octonion has a non-zero l part")
    return o[:4].copy()


# --------------------------------------------------------------------------
# Matrices (Sec. 2.2, Sec. 4)
# --------------------------------------------------------------------------


def omatmul(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Octonion matrix product (8, M, T) x (8, T, N): (X Y)_ij = sum_t X_it Y_tj."""
    return omul(X[:, :, :, None], Y[:, None, :, :]).sum(axis=2)


def omatmul_lr(*Xs: np.ndarray) -> np.ndarray:
    """Product of several octonion matrices read left to right, ((X Y) Z) ..."""
    acc = Xs[0]
    for X in Xs[1:]:
        acc = omatmul(acc, X)
    return acc


def omat_conj_transpose(X: np.ndarray) -> np.ndarray:
    """X^*: the transpose with every entry conjugated."""
    return oconj(np.swapaxes(X, 1, 2))


def eye(n: int) -> np.ndarray:
    """Octonion identity matrix I_n."""
    out = np.zeros((8, n, n))
    out[0] = np.eye(n)
    return out


def dft_matrix(p: int) -> np.ndarray:
    """Normalised DFT matrix F_p = (omega^((r-1)(c-1)) / sqrt(p)), omega =
    exp(-2 pi i / p) (eq. DFT), as a complex (p, p) array."""
    r = np.arange(p)
    return np.exp(-2j * np.pi * np.outer(r, r) / p) / np.sqrt(p)


def perm_matrix(p: int) -> np.ndarray:
    """P_p of eq. Pp: P_11 = 1 and P_rc = 1 where r + c = p + 2 (1-based)."""
    P = np.zeros((p, p))
    P[0, 0] = 1.0
    for r in range(2, p + 1):
        P[r - 1, p + 2 - r - 1] = 1.0
    return P


def times_unit(F: np.ndarray, u: np.ndarray) -> np.ndarray:
    """The octonion matrix F u (entries F_rc u, complex F_rc times the octonion u)."""
    return omul(from_complex(F), u.reshape((8,) + (1,) * F.ndim))


def kron_eye(O: np.ndarray, m: int) -> np.ndarray:
    """O (x) I_m (eq. kronecker) for an octonion matrix O (8, p, q)."""
    _, p, q = O.shape
    out = np.zeros((8, p * m, q * m))
    for r in range(p):
        for c in range(q):
            for t in range(m):
                out[:, r * m + t, c * m + t] = O[:, r, c]
    return out


UNITS = {
    "l": unit("l"),
    "jl": unit("jl"),
    "(l+jl)/sqrt2": (unit("l") + unit("jl")) / np.sqrt(2.0),
}


def diag_matrix(O: np.ndarray) -> np.ndarray:
    """The block diagonal octonion matrix Diag(Q) (eq. blockdiag) of a tensor
    given as octonions (8, m, n, p): block k is the frontal slice k."""
    _, m, n, p = O.shape
    out = np.zeros((8, m * p, n * p))
    for k in range(p):
        out[:, k * m:(k + 1) * m, k * n:(k + 1) * n] = O[..., k]
    return out


def diag_blocks(D: np.ndarray, m: int, n: int, p: int):
    """Inverse of ``diag_matrix``: the p diagonal blocks (8, m, n, p) and the
    largest magnitude found off the diagonal blocks."""
    blocks = np.stack([D[:, k * m:(k + 1) * m, k * n:(k + 1) * n] for k in range(p)], axis=-1)
    mask = np.ones(D.shape[1:], dtype=bool)
    for k in range(p):
        mask[k * m:(k + 1) * m, k * n:(k + 1) * n] = False
    off = float(np.max(np.abs(D[:, mask]), initial=0.0))
    return blocks, off


def bcirc_oct(Q: np.ndarray) -> np.ndarray:
    """bcirc of a quaternion tensor (4, m, n, p) as an octonion matrix
    (eq. circulant: block (r, c) is the slice (r - c) mod p, 0-based)."""
    _, m, n, p = Q.shape
    out = np.zeros((8, m * p, n * p))
    for r in range(p):
        for c in range(p):
            out[:4, r * m:(r + 1) * m, c * n:(c + 1) * n] = Q[:, :, :, (r - c) % p]
    return out


# --------------------------------------------------------------------------
# Theorem 4.4 and Theorem 5.1 in the octonion domain
# --------------------------------------------------------------------------


def block_diagonalize(Q: np.ndarray, u: np.ndarray):
    """(O (x) I_m) bcirc(Q) (O^* (x) I_n) with O = F_p u (Thm 4.3, Thm 4.4),
    read left to right.  Returns the diagonal blocks as quaternions
    (4, m, n, p) and the largest off-diagonal magnitude."""
    _, m, n, p = Q.shape
    O = times_unit(dft_matrix(p), u)
    L = kron_eye(O, m)
    R = kron_eye(omat_conj_transpose(O), n)
    D = omatmul_lr(L, bcirc_oct(Q), R)
    blocks, off = diag_blocks(D, m, n, p)
    return to_quat(blocks), off


def tprod_octonion(A: np.ndarray, B: np.ndarray, u: np.ndarray | None = None) -> np.ndarray:
    """The T-product A * B along the route of Theorem 5.1, every transform an
    octonion matrix product (no FFT).

    eq. A / eq. B: Diag(A_hat) = (F_p u (x) I_m) bcirc(A) (-F_p u (x) I_n), the
    same for B (O^* = -O, proof of Thm 4.1); A_hat = A_hat_1 + A_hat_2 j.
    eqs. C, C2, with Kronecker products of the permutation P_p of eq. Pp:
      Diag(C_hat_1) = (P (x) I_m) Diag(A_hat_1) Diag(B_hat_1) (P (x) I_s)
                      - Diag(conj A_hat_2) (P (x) I_n) Diag(B_hat_2) (P (x) I_s)
      Diag(C_hat_2) = (P (x) I_m) Diag(conj A_hat_1) (P (x) I_n) Diag(B_hat_2)
                      + Diag(A_hat_2) Diag(B_hat_1)
    eq. T-product-quaternion: bcirc(C) = (F_p^* u (x) I_m) Diag(C_hat)
    (-F_p^* u (x) I_s), read left to right; C is its first block column.
    The paper states the theorem for u = l.
    """
    if u is None:
        u = UNITS["l"]
    _, m, n, p = A.shape
    s = B.shape[2]
    Ah, offa = block_diagonalize(A, u)
    Bh, offb = block_diagonalize(B, u)
    scale = max(1.0, float(np.max(np.abs(A))) * p, float(np.max(np.abs(B))) * p)
    if max(offa, offb) > 1e-9 * scale:
        raise ValueError("bcirc not block diagonalized")
    Ah1, Ah2 = Ah[0] + 1j * Ah[1], Ah[2] + 1j * Ah[3]
    Bh1, Bh2 = Bh[0] + 1j * Bh[1], Bh[2] + 1j * Bh[3]

    def bdiag(X):   # complex (r, c, p) -> block diagonal complex matrix
        r, c, _ = X.shape
        out = np.zeros((r * p, c * p), dtype=complex)
        for k in range(p):
            out[k * r:(k + 1) * r, k * c:(k + 1) * c] = X[:, :, k]
        return out

    P = perm_matrix(p)
    Pm, Pn, Ps = np.kron(P, np.eye(m)), np.kron(P, np.eye(n)), np.kron(P, np.eye(s))
    C1 = Pm @ bdiag(Ah1) @ bdiag(Bh1) @ Ps - bdiag(np.conj(Ah2)) @ (Pn @ bdiag(Bh2) @ Ps)
    C2 = (Pm @ bdiag(np.conj(Ah1)) @ Pn) @ bdiag(Bh2) + bdiag(Ah2) @ bdiag(Bh1)
    Dc = np.zeros((8, m * p, s * p))
    Dc[0], Dc[1], Dc[2], Dc[3] = C1.real, C1.imag, C2.real, C2.imag
    Fs = times_unit(np.conj(dft_matrix(p)).T, u)
    bc = omatmul_lr(kron_eye(Fs, m), Dc, -kron_eye(Fs, s))
    bcq = to_quat(bc)
    return np.stack([bcq[:, k * m:(k + 1) * m, 0:s] for k in range(p)], axis=-1)
