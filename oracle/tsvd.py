"""FP64 T-SVD of a third-order quaternion tensor under the T-product of the
paper (a downstream method it names in Sec. 6; the decomposition itself is
not in the paper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` and ``bench.py``'s CPU legs use
this module; it shares no code with the CUDA path.

What is computed
----------------
For A in Q^{m x n x p} (layout (4, m, n, p) of ``oracle.qtp_oracle``) and
k = min(m, n): U in Q^{m x k x p}, S in Q^{k x k x p} f-diagonal (every
frontal slice diagonal, no j part), V in Q^{n x k x p} with

    A = U * S * V^H,   U^H * U = I_k,   V^H * V = I_k

(* the T-product, ^H the Kilmer-Martin conjugate transpose, I_k the identity
tensor), and sigma (p, k): the real diagonals of S's spectra.

Route (the per-frequency structure of Thm 5.1 in its plain-transform form):
with the unnormalised transforms A1_hat = fft(A1), A2_hat = fft(A2) along
mode 3 and g = (-f) mod p, the 2m x 2n complex matrix

    M_f(A) = [[A1_hat(f),           A2_hat(f)         ],
              [-conj(A2_hat(g)),    conj(A1_hat(g))   ]]

satisfies M_f(A * B) = M_f(A) M_f(B) (the products of Thm 5.1),
M_f(A^H) = M_f(A)^H, and M_g(A) = Q conj(M_f(A)) Q^T with Q = [[0, I], [-I, 0]].
So U, S, V follow from one SVD M_f = W diag(s) Z^H per frequency pair
{f, g}, its factors split by the same block pattern:

* f != g: W's columns of odd rank (1st, 3rd, ...) are U's spectra at f,
  those of even rank give U's spectra at g (through the conjugate block
  pattern); the same for Z and V; sigma(f) = s[0::2], sigma(g) = s[1::2].
* f == g (f = 0, and f = p / 2 for even p): M_f is the complex adjoint of a
  quaternion matrix, its singular values come in equal pairs, and the
  factors must keep the pattern: W's second half is Q^T conj(first half)
  (a quaternion SVD).  The first half takes one vector per pair, projected
  off the vectors already chosen and their partners.

Reading: the paper defines no T-SVD; the split of each pair's 2k singular
values into odd and even ranks is a convention chosen here (it makes the
tubal-rank-r truncation keep the 2r largest singular values of every M_f,
the best rank-2r approximation of each).

Parity pins (``tests/test_oracle_tsvd.py``): reconstruction, orthogonality
and f-diagonality checked with the T-product by its definition
(``tprod_def``, no FFT), Parseval's identity for sigma, the truncation error
in closed form and against other tubal-rank-r approximations, the real
special case against the real t-SVD (numpy SVD of the FFT slices), and p = 1
against the quaternion matrix SVD's paired singular values.
"""
from __future__ import annotations

import numpy as np

from .qtp_oracle import cd_join, cd_split


def _Q(k: int) -> np.ndarray:
    return np.block([[np.zeros((k, k)), np.eye(k)], [-np.eye(k), np.zeros((k, k))]])


def partner(X: np.ndarray) -> np.ndarray:
    """Q^T conj(X) for a (2k, c) block of columns: the quaternion partner of
    each column (the second half of a complex adjoint's columns)."""
    k = X.shape[0] // 2
    return _Q(k).T @ np.conj(X)


def spectral_matrix(A: np.ndarray, f: int) -> np.ndarray:
    """M_f(A) of the module docstring (2m x 2n complex)."""
    p = A.shape[-1]
    g = (-f) % p
    A1, A2 = cd_split(A)
    H1, H2 = np.fft.fft(A1, axis=-1), np.fft.fft(A2, axis=-1)
    return np.block([[H1[..., f], H2[..., f]], [-np.conj(H2[..., g]), np.conj(H1[..., g])]])


def _structured_half(M: np.ndarray, W: np.ndarray, s: np.ndarray, Z: np.ndarray, k: int):
    """Self-paired frequency: k left vectors (one per equal pair of singular
    values) such that [Wa, partner(Wa)] is orthonormal, their right vectors
    and singular values.  Candidates are W's columns in rank order, each
    projected off the chosen vectors and their partners (two passes)."""
    rows = M.shape[0]
    Wa = np.zeros((rows, 0), dtype=complex)
    Za = np.zeros((M.shape[1], 0), dtype=complex)
    sa = []
    for j in range(W.shape[1]):
        if Wa.shape[1] == k:
            break
        w = W[:, j].copy()
        B = np.concatenate([Wa, partner(Wa)], axis=1)
        for _ in range(2):
            w -= B @ (B.conj().T @ w)
        nw = np.linalg.norm(w)
        if nw < 0.5:
            continue                      # the partner of a chosen vector
        w /= nw
        sig = float(np.real(np.vdot(w, M @ (M.conj().T @ w)))) ** 0.5 if s[j] > 0 else 0.0
        if sig > 1e-12 * max(s[0], 1e-300):
            z = M.conj().T @ w / sig
        else:                             # null space: a right vector off the chosen ones
            z = None
            Bz = np.concatenate([Za, partner(Za)], axis=1)
            for c in range(Z.shape[1] - 1, -1, -1):
                cand = Z[:, c].copy()
                for _ in range(2):
                    cand -= Bz @ (Bz.conj().T @ cand)
                if np.linalg.norm(cand) > 0.5:
                    z = cand / np.linalg.norm(cand)
                    break
            sig = 0.0
        Wa = np.concatenate([Wa, w[:, None]], axis=1)
        Za = np.concatenate([Za, z[:, None]], axis=1)
        sa.append(sig)
    return Wa, np.asarray(sa), Za


def tsvd(A: np.ndarray):
    """T-SVD (U, S, V, sigma) of A (4, m, n, p); see the module docstring."""
    _, m, n, p = A.shape
    k = min(m, n)
    A1, A2 = cd_split(A)
    H1, H2 = np.fft.fft(A1, axis=-1), np.fft.fft(A2, axis=-1)
    U1h = np.zeros((m, k, p), dtype=complex)
    U2h = np.zeros((m, k, p), dtype=complex)
    V1h = np.zeros((n, k, p), dtype=complex)
    V2h = np.zeros((n, k, p), dtype=complex)
    sigma = np.zeros((p, k))
    for f in range(p):
        g = (-f) % p
        if f > g:
            continue
        M = np.block([[H1[..., f], H2[..., f]], [-np.conj(H2[..., g]), np.conj(H1[..., g])]])
        W, s, Zh = np.linalg.svd(M, full_matrices=False)
        Z = Zh.conj().T
        if f == g:
            Wa, sa, Za = _structured_half(M, W, s, Z, k)
            Wb, sb, Zb = partner(Wa), sa, partner(Za)
        else:
            Wa, Wb, Za, Zb = W[:, 0::2], W[:, 1::2], Z[:, 0::2], Z[:, 1::2]
            sa, sb = s[0::2], s[1::2]
        # M_f(U) = [Wa Wb] = [[U1(f), U2(f)], [-conj U2(g), conj U1(g)]]
        U1h[..., f], U2h[..., f] = Wa[:m], Wb[:m]
        U2h[..., g], U1h[..., g] = -np.conj(Wa[m:]), np.conj(Wb[m:])
        V1h[..., f], V2h[..., f] = Za[:n], Zb[:n]
        V2h[..., g], V1h[..., g] = -np.conj(Za[n:]), np.conj(Zb[n:])
        sigma[f], sigma[g] = sa, sb
    U = cd_join(np.fft.ifft(U1h, axis=-1), np.fft.ifft(U2h, axis=-1))
    V = cd_join(np.fft.ifft(V1h, axis=-1), np.fft.ifft(V2h, axis=-1))
    S1h = np.zeros((k, k, p), dtype=complex)
    for f in range(p):
        S1h[np.arange(k), np.arange(k), f] = sigma[f]
    S = cd_join(np.fft.ifft(S1h, axis=-1), np.zeros((k, k, p), dtype=complex))
    return U, S, V, sigma


def truncate(U: np.ndarray, S: np.ndarray, V: np.ndarray, r: int):
    """The tubal-rank-r part (U[:, :r], S[:r, :r], V[:, :r]) of a T-SVD."""
    return U[:, :, :r], S[:, :r, :r], V[:, :, :r]


def truncation_error_sq(sigma: np.ndarray, r: int) -> float:
    """||A - A_r||_F^2 over the four real components, A_r = U_r * S_r * V_r^H:
    by Parseval, (1 / p) times the sum over f of the squared dropped sigma(f)."""
    p = sigma.shape[0]
    return float(np.sum(sigma[:, r:] ** 2) / p)
