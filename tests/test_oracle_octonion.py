"""Octonion-domain statements of Sec. 2.2 and Sec. 4 checked on the FP64 oracle.

The octonion product (``oracle.octonion.omul``) is pinned first: to the
paper's multiplication table (tests/golden/octonion_units.json), to the
Cayley-Dickson doubling of the (separately pinned) Hamilton product, and to the
identities every octonion algebra satisfies (composition law, alternativity,
Moufang).  Then every proposition and theorem of Sec. 4 that the fast
T-product rests on is checked numerically on seeded random inputs, and the
whole octonion route of Theorem 5.1 against the T-product definition.

Unbracketed products are read left to right (the reading under which every
statement below holds; the module docstring of ``oracle.octonion`` gives it).
"""
import json
import os

import numpy as np
import pytest

import oracle as Q
from oracle import octonion as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = 1e-12


def rand_o(rng, *shape):
    return rng.standard_normal((8,) + shape)


def rand_c(rng, n=None):
    if n is None:
        return complex(*rng.standard_normal(2))
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def lr(*xs):
    acc = xs[0]
    for x in xs[1:]:
        acc = O.omul(acc, x)
    return acc


L, JL = O.unit("l"), O.unit("jl")
J = O.unit("j")


def c(z):           # complex p = a + b i as an octonion
    return O.from_complex(z)


def cj(z):          # p j
    return O.omul(c(z), J)


def cl(z):          # p l
    return O.omul(c(z), L)


def cjl(z):         # p (jl)
    return O.omul(c(z), JL)


def close(x, y, tol=TOL):
    return np.max(np.abs(np.asarray(x) - np.asarray(y))) <= tol * max(1.0, float(np.max(np.abs(y))))


# ------------------------------------------------------------- the product


def test_octonion_table_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "octonion_units.json")))
    assert tuple(g["basis"]) == O.BASIS
    seen = 0
    for x, row in g["products"].items():
        for y, (sign, u) in row.items():
            np.testing.assert_array_equal(O.omul(O.unit(x), O.unit(y)), sign * O.unit(u), err_msg=f"{x}*{y}")
            seen += 1
    assert seen == 64


def test_octonion_is_cayley_dickson_doubling_of_hamilton():
    """(q1 + q2 l)(q3 + q4 l) = (q1 q3 - conj(q4) q2) + (q4 q1 + q2 conj(q3)) l,
    the doubling that gives the octonions from the quaternions (Sec. 2.2's
    quaternionic form o = q1 + q2 l), built on the Hamilton product."""
    rng = np.random.default_rng(11)
    x, y = rand_o(rng, 50), rand_o(rng, 50)
    q1, q2, q3, q4 = x[:4], x[4:], y[:4], y[4:]
    H, cq = Q.hamilton, Q.qconj
    want = np.concatenate([H(q1, q3) - H(cq(q4), q2), H(q4, q1) + H(q2, cq(q3))])
    np.testing.assert_allclose(O.omul(x, y), want, rtol=0, atol=1e-13)


def test_quaternion_subalgebra_is_hamilton():
    rng = np.random.default_rng(12)
    a, b = rng.standard_normal((4, 40)), rng.standard_normal((4, 40))
    got = O.omul(O.from_quat(a), O.from_quat(b))
    np.testing.assert_allclose(got[:4], Q.hamilton(a, b), rtol=0, atol=1e-13)
    assert np.all(got[4:] == 0)


def test_composition_conjugation_alternativity_moufang():
    rng = np.random.default_rng(13)
    x, y, z = rand_o(rng, 64), rand_o(rng, 64), rand_o(rng, 64)
    m = O.omul
    np.testing.assert_allclose(O.onorm(m(x, y)), O.onorm(x) * O.onorm(y), rtol=1e-13)
    np.testing.assert_allclose(O.oconj(m(x, y)), m(O.oconj(y), O.oconj(x)), atol=1e-13)
    xx = m(O.oconj(x), x)
    np.testing.assert_allclose(xx[0], O.onorm(x) ** 2, rtol=1e-13)
    np.testing.assert_allclose(xx[1:], 0, atol=1e-13)
    np.testing.assert_allclose(m(m(x, x), y), m(x, m(x, y)), atol=1e-12)    # left alternative
    np.testing.assert_allclose(m(y, m(x, x)), m(m(y, x), x), atol=1e-12)    # right alternative
    np.testing.assert_allclose(m(m(x, y), x), m(x, m(y, x)), atol=1e-12)    # flexible
    np.testing.assert_allclose(m(z, m(x, m(z, y))), m(m(m(z, x), z), y), atol=1e-11)  # Moufang
    # but neither associative nor commutative in general
    assert np.min(np.max(np.abs(m(m(x, y), z) - m(x, m(y, z))), axis=0)) > 1e-3
    assert np.min(np.max(np.abs(m(x, y) - m(y, x)), axis=0)) > 1e-3


def test_sec41_examples_non_commutative_non_associative():
    i, j, l = O.unit("i"), O.unit("j"), O.unit("l")
    assert not np.array_equal(O.omul(i, j), O.omul(j, i))
    assert not np.array_equal(O.omul(i, O.unit("jl")), O.omul(O.omul(i, j), l))


def test_l_conjugates_quaternions():
    """l q = conj(q) l for every quaternion q, and (s l)(t l) is a quaternion
    (the two facts Sec. 4 opens with)."""
    rng = np.random.default_rng(14)
    q = O.from_quat(rng.standard_normal((4, 30)))
    s, t = O.from_quat(rng.standard_normal((4, 30))), O.from_quat(rng.standard_normal((4, 30)))
    l = L.reshape(8, 1)
    np.testing.assert_allclose(O.omul(l, q), O.omul(O.oconj(q), l), atol=1e-13)
    st = O.omul(O.omul(s, l), O.omul(t, l))
    np.testing.assert_allclose(st[4:], 0, atol=1e-13)


# ------------------------------------------------------------- Prop 4.1


@pytest.mark.parametrize("seed", range(5))
def test_prop41(seed):
    rng = np.random.default_rng(100 + seed)
    p, q, r, s = (rand_c(rng) for _ in range(4))
    cg = np.conj
    # (i) (p + q j)[(r + s j) l] = [(r + s j) l] conj(p + q j)
    pq = c(p) + cj(q)
    rsl = O.omul(c(r) + cj(s), L)
    assert close(O.omul(pq, rsl), O.omul(rsl, O.oconj(pq)))
    # (ii) (pl) q (rl) = -p conj(q) conj(r) = [p(jl)] q [r(jl)]
    want = c(-p * cg(q) * cg(r))
    assert close(lr(cl(p), c(q), cl(r)), want)
    assert close(lr(cjl(p), c(q), cjl(r)), want)
    # (iii) (pl)(qj)(rl) = p q conj(r) j = [p(jl)](qj)[r(jl)]
    want = cj(p * q * cg(r))
    assert close(lr(cl(p), cj(q), cl(r)), want)
    assert close(lr(cjl(p), cj(q), cjl(r)), want)
    # (iv) (pl) q [r(jl)] = conj(p) q conj(r) j = -[p(jl)] q (rl)
    want = cj(cg(p) * q * cg(r))
    assert close(lr(cl(p), c(q), cjl(r)), want)
    assert close(-lr(cjl(p), c(q), cl(r)), want)
    # (v) (pl)(qj)[r(jl)] = conj(p q r) = -[p(jl)](qj)(rl)
    want = c(cg(p) * cg(q) * cg(r))
    assert close(lr(cl(p), cj(q), cjl(r)), want)
    assert close(-lr(cjl(p), cj(q), cl(r)), want)


def test_prop41_needs_left_to_right_reading():
    """Grouping the other way breaks (iii): the reading is not a matter of taste."""
    rng = np.random.default_rng(7)
    p, q, r = (rand_c(rng) for _ in range(3))
    right = O.omul(cl(p), O.omul(cj(q), cl(r)))
    assert not close(right, cj(p * q * np.conj(r)), 1e-6)


def test_remark41_special_commutative_rule():
    """p (q l) = (q l) conj(p) for quaternions p, q; p (q l) != conj(q l) p in general."""
    rng = np.random.default_rng(15)
    p = O.from_quat(rng.standard_normal((4, 20)))
    ql = O.omul(O.from_quat(rng.standard_normal((4, 20))), L.reshape(8, 1))
    np.testing.assert_allclose(O.omul(p, ql), O.omul(ql, O.oconj(p)), atol=1e-13)
    assert np.min(np.max(np.abs(O.omul(p, ql) - O.omul(O.oconj(ql), p)), axis=0)) > 1e-3


@pytest.mark.parametrize("u", list(O.UNITS))
def test_eq_relation_remark(u):
    """(p u)(q + r j)(s u) = -p conj(q) conj(s) + p r conj(s) j for complex p, q, r, s."""
    rng = np.random.default_rng(16)
    uu = O.UNITS[u].reshape(8, 1)
    p, q, r, s = (rand_c(rng, 25) for _ in range(4))
    lhs = lr(O.omul(c(p), uu), c(q) + cj(r), O.omul(c(s), uu))
    rhs = c(-p * np.conj(q) * np.conj(s)) + cj(p * r * np.conj(s))
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


# ------------------------------------------------------------- Prop 4.2


@pytest.mark.parametrize("seed", range(5))
def test_prop42(seed):
    rng = np.random.default_rng(200 + seed)
    p, q, r, s, t = (rand_c(rng) for _ in range(5))
    cg = np.conj
    m = O.omul
    # (i)
    assert close(m(c(p), lr(cl(q), c(r), cl(s))), lr(c(p), cl(q), c(r), cl(s)))
    assert close(m(c(p), lr(cl(q), cj(r), cl(s))), lr(c(p), cl(q), cj(r), cl(s)))
    # (ii)
    assert close(m(cj(p), lr(cl(q), c(r), cl(s))), lr(cj(p), cl(cg(q)), c(r), cl(cg(s))))
    assert close(m(cj(p), lr(cl(q), cj(r), cl(s))), lr(cj(p), cl(cg(q)), cj(r), cl(cg(s))))
    # (iii)
    assert close(lr(cl(p), lr(cl(q), c(r), cl(s)), cl(t)), lr(m(cl(p), cl(q)), c(r), m(cl(s), cl(t))))
    assert close(lr(cl(p), lr(c(q), c(r), c(s)), cl(t)), lr(m(cl(p), c(q)), c(r), m(c(s), cl(t))))
    # (iv), first identity
    assert close(lr(cl(p), lr(cl(q), cj(r), cl(s)), cl(t)),
                 lr(m(cl(p), cl(cg(q))), cj(r), m(cl(s), cl(cg(t)))))
    # (v)
    assert close(lr(cl(p), cl(q), cl(r)), m(cl(p), m(cl(q), cl(r))))
    assert close(lr(cjl(p), cl(q), cl(r)), m(cjl(p), m(cl(cg(q)), cl(cg(r)))))
    # (vi)
    assert close(lr(cl(t), c(p) + cj(q), c(r) + cj(s)),
                 m(cl(t), c(p * r - cg(q) * s) + cj(cg(p) * s + q * r)))


def test_prop42_iv_second_identity_reading():
    """(pl)[c (rj) d](sl) = [(pl) c](rj)[d (sl)]: c and d are not defined in the
    statement.  It holds for real c, d; for complex c, d it needs conj(c) on
    the right-hand side (both recorded here, the complex form as it fails)."""
    rng = np.random.default_rng(17)
    p, r, s = (rand_c(rng) for _ in range(3))
    m = O.omul
    cr, dr = rng.standard_normal(2)
    assert close(lr(cl(p), lr(c(cr), cj(r), c(dr)), cl(s)), lr(m(cl(p), c(cr)), cj(r), m(c(dr), cl(s))))
    cc, dc = rand_c(rng), rand_c(rng)
    lhs = lr(cl(p), lr(c(cc), cj(r), c(dc)), cl(s))
    assert not close(lhs, lr(m(cl(p), c(cc)), cj(r), m(c(dc), cl(s))), 1e-6)
    assert close(lhs, lr(m(cl(p), c(np.conj(cc))), cj(r), m(c(dc), cl(s))))


def test_remark43_non_associative_cases():
    rng = np.random.default_rng(18)
    p, q, r, s, t = (rand_c(rng) for _ in range(5))
    m = O.omul
    pairs = [
        (lr(cl(p), cl(q), cj(r)), m(cl(p), m(cl(q), cj(r)))),
        (lr(cj(p), cl(q), cl(r)), m(cj(p), m(cl(q), cl(r)))),
        (lr(cjl(p), cl(q), cl(r)), m(cjl(p), m(cl(q), cl(r)))),
        (lr(cl(t), c(p) + cj(q), c(r) + cj(s)), m(cl(t), m(c(p) + cj(q), c(r) + cj(s)))),
    ]
    for a, b in pairs:
        assert not close(a, b, 1e-6)


# ------------------------------------------------------------- Thm 4.1


def test_eq_FpFp_and_Pp():
    for p in range(1, 10):
        F = O.dft_matrix(p)
        P = O.perm_matrix(p)
        np.testing.assert_allclose(F @ F, P, atol=1e-13)
        np.testing.assert_allclose(F.conj().T @ F.conj().T, P, atol=1e-13)
        np.testing.assert_allclose(F @ F.conj().T, np.eye(p), atol=1e-13)
        Fl, Fsl = O.times_unit(F, L), O.times_unit(F.conj().T, L)
        want = O.from_complex(P)
        np.testing.assert_allclose(-O.omatmul(Fl, Fsl), want, atol=1e-13)
        np.testing.assert_allclose(-O.omatmul(Fsl, Fl), want, atol=1e-13)


@pytest.mark.parametrize("u", list(O.UNITS))
def test_thm41_unitary(u):
    for p in range(1, 10):
        Om = O.times_unit(O.dft_matrix(p), O.UNITS[u])
        Os = O.omat_conj_transpose(Om)
        np.testing.assert_allclose(Os, -Om, atol=1e-15)
        np.testing.assert_allclose(O.omatmul(Om, Os), O.eye(p), atol=1e-13)
        np.testing.assert_allclose(O.omatmul(Os, Om), O.eye(p), atol=1e-13)


# ------------------------------------------------------------- Thm 4.2


def circ_oct(q):
    """circ(q_1, ..., q_p) of quaternions (4, p) as an octonion matrix (eq. circulant)."""
    return O.bcirc_oct(q[:, None, None, :])


def fft_conj_vec(q):
    """q_hat = fft(conj q1) - fft(q2) j (eq. fft-q), by numpy's FFT."""
    q1, q2 = q[0] + 1j * q[1], q[2] + 1j * q[3]
    h1, h2 = np.fft.fft(np.conj(q1)), -np.fft.fft(q2)
    return np.stack([h1.real, h1.imag, h2.real, h2.imag])


@pytest.mark.parametrize("u", list(O.UNITS))
def test_thm42_diagonalizes_circulant_quaternion(u):
    rng = np.random.default_rng(300)
    for p in range(1, 10):
        q = rng.standard_normal((4, p))
        Om = O.times_unit(O.dft_matrix(p), O.UNITS[u])
        D = O.omatmul_lr(Om, circ_oct(q), O.omat_conj_transpose(Om))
        diag = D[:, np.arange(p), np.arange(p)]
        off = D.copy()
        off[:, np.arange(p), np.arange(p)] = 0
        assert np.max(np.abs(off)) < 1e-12, (u, p)
        assert np.max(np.abs(diag[4:])) < 1e-12               # stays in the quaternions (Remark 4.4 (i))
        # q_hat = sqrt(p) F_p conj(q): complex entries times quaternions, as octonions
        qbar = O.oconj(O.from_quat(q))
        want = O.omatmul(O.from_complex(np.sqrt(p) * O.dft_matrix(p)), qbar[:, :, None])[:, :, 0]
        np.testing.assert_allclose(diag, want, atol=1e-12)
        np.testing.assert_allclose(diag[:4], fft_conj_vec(q), atol=1e-12)


def test_complex_dft_does_not_diagonalize_quaternion_circulants():
    """Sec. 3's negative result in this module's arithmetic: F_p (u = 1) and F_p j
    leave off-diagonal entries for p >= 3 once q has a j part."""
    rng = np.random.default_rng(301)
    for p in range(3, 8):
        q = rng.standard_normal((4, p))
        for u in (O.unit("1"), J):
            Om = O.times_unit(O.dft_matrix(p), u)
            D = O.omatmul_lr(Om, circ_oct(q), O.omat_conj_transpose(Om))
            D[:, np.arange(p), np.arange(p)] = 0
            assert np.max(np.abs(D)) > 1e-3


@pytest.mark.parametrize("u", list(O.UNITS))
def test_remark42_iii_inverse(u):
    """O = F_p^* u: circ(q) = O Diag(q_hat) O^* gives q = ifft(conj q_hat_1) - ifft(q_hat_2) j."""
    rng = np.random.default_rng(302)
    for p in range(1, 9):
        qh = rng.standard_normal((4, p))
        Om = O.times_unit(O.dft_matrix(p).conj().T, O.UNITS[u])
        Dq = np.zeros((8, p, p))
        Dq[:4, np.arange(p), np.arange(p)] = qh
        M = O.omatmul_lr(Om, Dq, O.omat_conj_transpose(Om))
        h1, h2 = qh[0] + 1j * qh[1], qh[2] + 1j * qh[3]
        q1, q2 = np.fft.ifft(np.conj(h1)), -np.fft.ifft(h2)
        q = np.stack([q1.real, q1.imag, q2.real, q2.imag])
        np.testing.assert_allclose(M, circ_oct(q), atol=1e-12)


# ------------------------------------------------------------- Thm 4.3 / 4.4


@pytest.mark.parametrize("u", list(O.UNITS))
@pytest.mark.parametrize("m,n,p", [(1, 1, 1), (2, 3, 4), (3, 2, 5), (2, 2, 7)])
def test_thm43_44_block_diagonalization(u, m, n, p):
    rng = np.random.default_rng(400 + m * 100 + n * 10 + p)
    Qt = rng.standard_normal((4, m, n, p))
    Qh, off = O.block_diagonalize(Qt, O.UNITS[u])
    assert off < 1e-12
    # eq. fft-Q: fft(conj Q1) - fft(Q2) j along mode 3
    Q1, Q2 = Q.cd_split(Qt)
    h1, h2 = np.fft.fft(np.conj(Q1), axis=-1), -np.fft.fft(Q2, axis=-1)
    np.testing.assert_allclose(Qh, Q.cd_join(h1, h2), atol=1e-12)
    # eq. relation-unfold: unfold(Q_hat) = sqrt(p) (F_p (x) I_m) unfold(conj Q)
    K = O.from_complex(np.sqrt(p) * np.kron(O.dft_matrix(p), np.eye(m)))
    got = O.omatmul(K, O.from_quat(Q.unfold(Q.qconj(Qt))))
    np.testing.assert_allclose(got[:4], Q.unfold(Qh), atol=1e-12)


@pytest.mark.parametrize("u", list(O.UNITS))
def test_remark44_iii_inversion(u):
    """Inverting the block diagonalization with F_p^* u alone fails (non-
    associativity); eq. ifftA's two-term form recovers bcirc(Q)."""
    rng = np.random.default_rng(500)
    m, n, p = 2, 3, 5
    Qt = rng.standard_normal((4, m, n, p))
    uu = O.UNITS[u]
    Qh, _ = O.block_diagonalize(Qt, uu)
    F, Fs = O.times_unit(O.dft_matrix(p), uu), O.times_unit(O.dft_matrix(p).conj().T, uu)
    Dfull = O.diag_matrix(O.from_quat(Qh))
    naive = O.omatmul_lr(O.kron_eye(Fs, m), O.bcirc_oct(Qt), -O.kron_eye(Fs, n))
    assert np.max(np.abs(naive - Dfull)) > 1e-3
    D1 = Dfull.copy()
    D1[2:] = 0                                  # Diag(Q_hat_1)
    D2j = Dfull.copy()
    D2j[:2] = 0
    D2j[4:] = 0                                 # Diag(Q_hat_2) j
    bc = (O.omatmul_lr(-O.kron_eye(F, m), D1, O.kron_eye(F, n))
          + O.omatmul_lr(-O.kron_eye(Fs, m), D2j, O.kron_eye(Fs, n)))
    np.testing.assert_allclose(bc, O.bcirc_oct(Qt), atol=1e-12)


# ------------------------------------------------------------- Thm 5.1


@pytest.mark.parametrize("u", list(O.UNITS))
@pytest.mark.parametrize("m,n,s,p", [(1, 1, 1, 1), (2, 3, 2, 4), (2, 2, 3, 5), (1, 2, 1, 3), (3, 2, 2, 6),
                                     (1, 1, 1, 2)])
def test_thm51_octonion_route_is_the_t_product(u, m, n, s, p):
    """bcirc(C) from eqs. A, B, C, C2 and eq. T-product-quaternion, all in
    octonion matrix arithmetic, equals the T-product by its definition (and
    the oracle's FFT form of Algorithm 5.1)."""
    rng = np.random.default_rng(600 + m + 10 * n + 100 * s + 1000 * p)
    A = rng.standard_normal((4, m, n, p))
    B = rng.standard_normal((4, n, s, p))
    C = O.tprod_octonion(A, B, O.UNITS[u])
    np.testing.assert_allclose(C, Q.tprod_def(A, B), atol=1e-11)
    np.testing.assert_allclose(C, Q.alg51(A, B), atol=1e-11)


def test_to_quat_rejects_l_part():
    with pytest.raises(ValueError):
        O.to_quat(O.unit("il"))
