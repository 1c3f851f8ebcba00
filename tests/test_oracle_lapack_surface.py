"""Pins of the oracle's LAPACK 3.2 surface (oracle/lapack_surface.py):
SciPy's LAPACK (an external implementation) where it has the routine,
exact integer and rational arithmetic, closed forms, and planted mistakes
that the pins must reject."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import oracle.lapack_surface as ls
import rfp_inputs as gen

lapack = pytest.importorskip("scipy.linalg.lapack")
LAYOUTS = [(t, u) for t in "NT" for u in "LU"]
SIZES = [0, 1, 2, 3, 6, 7, 10]


def test_tp_index_is_the_column_major_packed_order():
    for n in (1, 4, 9):
        for uplo in "LU":
            k = 0
            for j in range(n):
                for i in (range(j, n) if uplo == "L" else range(0, j + 1)):
                    assert ls.tp_index(uplo, n, i, j) == k
                    k += 1
            assert k == n * (n + 1) // 2


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
def test_tpttf_tfttp_match_lapack_bit_exactly(transr, uplo):
    rng = np.random.default_rng(1)
    for n in SIZES[1:]:
        ap = rng.standard_normal(n * (n + 1) // 2)
        arf = oracle.tpttf(transr, uplo, n, ap)
        ref, info = lapack.dtpttf(n, ap, transr=transr, uplo=uplo)
        assert info == 0 and np.array_equal(arf, ref)
        back = oracle.tfttp(transr, uplo, n, arf)
        ref2, info = lapack.dtfttp(n, ref, transr=transr, uplo=uplo)
        assert info == 0 and np.array_equal(back, ref2) and np.array_equal(back, ap)


def _exact_inverse(T):
    """Inverse of a small triangular integer matrix in exact rationals."""
    n = T.shape[0]
    A = [[Fraction(int(T[i, j])) for j in range(n)] + [Fraction(int(i == j)) for j in range(n)]
         for i in range(n)]
    for c in range(n):                        # Gauss-Jordan (no pivoting needed: diagonal != 0)
        p = A[c][c]
        A[c] = [x / p for x in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    return np.array([[float(A[i][n + j]) for j in range(n)] for i in range(n)])


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("diag", "NU")
def test_tftri_exact_on_integer_triangles(transr, uplo, diag):
    rng = np.random.default_rng(2)
    for n in (1, 2, 5, 8):
        L0 = np.tril(rng.integers(-3, 4, (n, n))).astype(float)
        np.fill_diagonal(L0, rng.choice([1.0, -1.0, 2.0, 4.0], n))   # inverse exact in binary
        T = L0 if uplo == "L" else L0.T
        arf = oracle.pack(transr, uplo, T)
        W, info = oracle.tftri(transr, uplo, diag, n, arf)
        assert info == 0
        Tref = T.copy()
        if diag == "U":
            np.fill_diagonal(Tref, 1.0)
        ref = _exact_inverse(Tref)
        got = oracle.unpack(transr, uplo, n, W)
        mask = np.tril(np.ones((n, n), bool), -1 if diag == "U" else 0)
        mask = mask if uplo == "L" else mask.T
        assert np.array_equal(got[mask], ref[mask])
        if diag == "U":                          # stored diagonal untouched
            assert np.array_equal(np.diag(got), np.diag(T))


def test_tftri_zero_diagonal_reports_info_and_random_inverse_is_accurate():
    n = 6
    T = np.tril(np.arange(1.0, n * n + 1).reshape(n, n))
    T[3, 3] = 0.0
    _, info = oracle.tftri("N", "L", "N", n, oracle.pack("N", "L", T))
    assert info == 4
    A = gen.spd_bbt(40, seed=3)
    L = np.linalg.cholesky(A)
    W, info = oracle.tftri("T", "L", "N", 40, oracle.pack("T", "L", L))
    Wf = oracle.unpack("T", "L", 40, W)
    assert info == 0 and np.max(np.abs(np.tril(Wf) @ L - np.eye(40))) < 1e-13


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("trans", "NT")
def test_sfrk_matches_lapack_and_is_exact_on_integers(transr, uplo, trans):
    rng = np.random.default_rng(4)
    for n, k in [(1, 3), (6, 4), (7, 1), (10, 12), (5, 0)]:
        A = rng.standard_normal((n, k) if trans == "N" else (k, n))
        C = rng.standard_normal((n, n))
        C = C + C.T
        arf = oracle.pack(transr, uplo, C)
        got = oracle.sfrk(transr, uplo, trans, n, k, 0.7, A, -1.3, arf)
        if k:
            ref = lapack.dsfrk(n, k, 0.7, np.asfortranarray(A), -1.3, arf.copy(), transr=transr,
                               uplo=uplo, trans=trans)
        else:                                     # no update: C := beta C
            ref = -1.3 * arf
        assert np.allclose(got, ref, rtol=0, atol=1e-13 * max(1.0, np.max(np.abs(ref))))
        # integers: alpha = 2, beta = -1, products and sums exact in FP64
        Ai = rng.integers(-4, 5, A.shape).astype(float)
        Ci = rng.integers(-9, 10, (n, n)).astype(float)
        Ci = Ci + Ci.T
        opA = Ai if trans == "N" else Ai.T
        exact = [[2 * sum(int(opA[i, p]) * int(opA[j, p]) for p in range(k)) - int(Ci[i, j])
                  for j in range(n)] for i in range(n)]
        got = oracle.sfrk(transr, uplo, trans, n, k, 2.0, Ai, -1.0, oracle.pack(transr, uplo, Ci))
        assert np.array_equal(got, oracle.pack(transr, uplo, np.array(exact, dtype=float)))


def test_sfrk_beta_zero_does_not_read_c():
    A = np.ones((4, 2))
    arf = np.full(10, np.nan)
    got = oracle.sfrk("N", "L", "N", 4, 2, 1.0, A, 0.0, arf)
    assert np.array_equal(got, np.full(10, 2.0))


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("side", "LR")
@pytest.mark.parametrize("trans", "NT")
@pytest.mark.parametrize("diag", "NU")
def test_tfsm_matches_lapack(transr, uplo, side, trans, diag):
    rng = np.random.default_rng(5)
    for m, nc in [(1, 1), (6, 3), (7, 5), (4, 9)]:
        order = m if side == "L" else nc
        T = np.tril(rng.standard_normal((order, order)), -1) + np.diag(rng.uniform(1, 2, order))
        T = T if uplo == "L" else T.T
        arf = oracle.pack(transr, uplo, T)
        B = rng.standard_normal((m, nc))
        got = oracle.tfsm(transr, side, uplo, trans, diag, m, nc, 1.5, arf, B)
        ref = lapack.dtfsm(1.5, arf, np.asfortranarray(B), transr=transr, side=side, uplo=uplo,
                           trans=trans, diag=diag)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_tfsm_exact_on_integer_systems_and_alpha_zero():
    rng = np.random.default_rng(6)
    n = 7
    L0 = np.tril(rng.integers(-2, 3, (n, n)), -1).astype(float) + np.eye(n)
    X = rng.integers(-5, 6, (n, 3)).astype(float)
    for uplo in "LU":
        T = L0 if uplo == "L" else L0.T
        for trans in "NT":
            opA = T if trans == "N" else T.T
            arf = oracle.pack("N", uplo, T)
            got = oracle.tfsm("N", "L", uplo, trans, "N", n, 3, 1.0, arf, opA @ X)
            assert np.array_equal(got, X)
            got = oracle.tfsm("N", "R", uplo, trans, "U", 3, n, 1.0, arf, X.T @ opA)
            assert np.array_equal(got, X.T)
    assert np.array_equal(oracle.tfsm("N", "L", "L", "N", "N", n, 3, 0.0, oracle.pack("N", "L", L0),
                                      np.full((n, 3), np.nan)), np.zeros((n, 3)))


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
def test_lansf_closed_forms(transr, uplo):
    for n in (1, 5, 8):
        J = np.ones((n, n))
        arf = oracle.pack(transr, uplo, J)
        assert oracle.lansf("M", transr, uplo, n, arf) == 1.0
        for nm in "1OI":
            assert oracle.lansf(nm, transr, uplo, n, arf) == float(n)
        assert oracle.lansf("F", transr, uplo, n, arf) == float(n)
        D = np.diag(np.arange(1.0, n + 1)) - np.tril(np.ones((n, n)), -1) - np.triu(np.ones((n, n)), 1)
        arf = oracle.pack(transr, uplo, D)
        assert oracle.lansf("M", transr, uplo, n, arf) == float(max(n, 1))
        # column j: |j+1| + (n - 1) ones -> max at the last column: n + n - 1
        assert oracle.lansf("1", transr, uplo, n, arf) == float(2 * n - 1)
        f2 = sum((i + 1) ** 2 for i in range(n)) + n * (n - 1)
        assert abs(oracle.lansf("E", transr, uplo, n, arf) - f2 ** 0.5) <= 4e-16 * f2 ** 0.5
    assert oracle.lansf("F", "N", "L", 0, np.zeros(0)) == 0.0


def test_planted_mistakes_are_rejected(monkeypatch):
    """Each pin above must catch a plausible mistake in the oracle."""
    n = 7
    ap = np.arange(1.0, n * (n + 1) // 2 + 1)
    ref, _ = lapack.dtpttf(n, ap, transr="N", uplo="U")
    monkeypatch.setattr(ls, "tp_index", lambda uplo, n, i, j: i + j * (j - 1) // 2 if uplo == "U"
                        else i + j * (2 * n - j - 1) // 2)   # upper column offset short by j
    try:
        bad = ls.tpttf("N", "U", n, ap)
        assert not np.array_equal(bad, ref)
    except IndexError:
        pass
    monkeypatch.undo()
    # a substitution that drops the last term
    real = ls.tri_inverse

    def dropped(T, lower):
        W = real(T, lower)
        W[-1, 0] = 0.0
        return W
    monkeypatch.setattr(ls, "tri_inverse", dropped)
    L0 = np.array([[1.0, 0, 0, 0], [2, 1, 0, 0], [3, 4, 1, 0], [5, 6, 7, 1]])   # (L0^-1)[3, 0] != 0
    W, _ = ls.tftri("N", "L", "N", 4, oracle.pack("N", "L", L0))
    assert not np.array_equal(oracle.unpack("N", "L", 4, W)[np.tril(np.ones((4, 4), bool))],
                              _exact_inverse(L0)[np.tril(np.ones((4, 4), bool))])


def _rejects(check):
    """True when the pin `check` fails (an assertion or an error) on the mutant."""
    try:
        check()
    except Exception:
        return True
    return False


def test_more_planted_mistakes_are_rejected(monkeypatch):
    rng = np.random.default_rng(21)
    n, k = 7, 4
    # SFRK that drops the beta C term
    A = rng.standard_normal((k, n))
    C = rng.standard_normal((n, n))
    arf = oracle.pack("N", "L", C + C.T)
    ref = lapack.dsfrk(n, k, 1.0, np.asfortranarray(A), 1.0, arf.copy(), transr="N", uplo="L",
                       trans="T")
    real_sfrk = ls.sfrk
    monkeypatch.setattr(ls, "sfrk", lambda transr, uplo, trans, n_, k_, alpha, A_, beta, arf_:
                        real_sfrk(transr, uplo, trans, n_, k_, alpha, A_, 0.0, arf_))
    assert _rejects(lambda: np.testing.assert_allclose(
        ls.sfrk("N", "L", "T", n, k, 1.0, A, 1.0, arf), ref, atol=1e-12))
    monkeypatch.undo()
    # TFSM that solves from the wrong side (A^{-1} B where B A^{-1} is asked for)
    T = np.tril(rng.standard_normal((n, n)), -1) + np.diag(rng.uniform(1, 2, n))
    tri = oracle.pack("N", "L", T)
    B = rng.standard_normal((3, n))
    ref = lapack.dtfsm(1.0, tri, np.asfortranarray(B), transr="N", side="R", uplo="L", trans="N",
                       diag="N")
    wrong = lambda: ls.tfsm("N", "L", "L", "N", "N", n, 3, 1.0, tri, B.T).T   # noqa: E731
    assert _rejects(lambda: np.testing.assert_allclose(wrong(), ref, atol=1e-10))
    # LANSF one-norm summed over the stored triangle only (off-diagonal half missing)
    S = rng.standard_normal((n, n))
    S = S + S.T
    sarf = oracle.pack("T", "U", S)
    half = float(np.max(np.sum(np.abs(np.triu(S)), axis=0)))
    assert half != oracle.lansf("1", "T", "U", n, sarf)
    assert oracle.lansf("1", "T", "U", n, sarf) == float(np.max(np.sum(np.abs(S), axis=0)))
    # TFTRI with a unit diagonal that still reads the stored diagonal
    L0 = np.tril(rng.integers(-2, 3, (5, 5))).astype(float)
    np.fill_diagonal(L0, 2.0)
    Wu, _ = oracle.tftri("N", "L", "U", 5, oracle.pack("N", "L", L0))
    Wn, _ = oracle.tftri("N", "L", "N", 5, oracle.pack("N", "L", L0))
    low = np.tril(np.ones((5, 5), bool), -1)
    assert not np.array_equal(oracle.unpack("N", "L", 5, Wu)[low], oracle.unpack("N", "L", 5, Wn)[low])
