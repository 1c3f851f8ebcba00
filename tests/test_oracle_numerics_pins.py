"""Pins for the oracle's FP64 factorization, solve and inverse, CPU only.

Closed forms whose exact answer is known (Pascal matrices, integer factors,
diagonal matrices, the second-difference matrix), a 50-digit brute force on
tiny inputs, the backward-error bounds of Higham's analysis that the paper's
stability section relies on, LAPACK's own RFP routines (SciPy), and the
failure index for matrices that are not positive definite.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
import rfp_inputs as gen
from rfp_inputs import LAYOUTS

EPS = np.finfo(np.float64).eps


def _factor_full(transr, uplo, n, arf):
    """Lower-triangular L from an RFP factor (U^T for UPLO='U')."""
    F = oracle.unpack(transr, uplo, n, arf)
    return np.tril(F) if uplo == "L" else np.triu(F).T


def _sym_full(transr, uplo, n, arf):
    F = oracle.unpack(transr, uplo, n, arf)
    return np.tril(F) + np.tril(F, -1).T if uplo == "L" else np.triu(F) + np.triu(F, 1).T


def _pftrf(transr, uplo, A):
    n = A.shape[0]
    out, info = oracle.pftrf(transr, uplo, n, oracle.pack(transr, uplo, A))
    return out, info


# ---- factorization -------------------------------------------------------

@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [1, 2, 7, 12, 19])
def test_pascal_factor_exact(transr, uplo, n):
    P, Lexact = gen.pascal(n)
    out, info = _pftrf(transr, uplo, P)
    assert info == 0
    np.testing.assert_array_equal(_factor_full(transr, uplo, n, out), Lexact)


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [3, 8, 33, 64])
def test_integer_factor_exact(transr, uplo, n):
    A, L0 = gen.spd_integer_factor(n, seed=n)
    out, info = _pftrf(transr, uplo, A)
    assert info == 0
    np.testing.assert_array_equal(_factor_full(transr, uplo, n, out), L0)


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
def test_diagonal_factor_correctly_rounded(transr, uplo):
    d = np.linspace(0.3, 17.0, 23)
    out, info = _pftrf(transr, uplo, np.diag(d))
    assert info == 0
    np.testing.assert_array_equal(_factor_full(transr, uplo, 23, out), np.diag(np.sqrt(d)))


def _decimal_cholesky(A):
    getcontext().prec = 50
    n = A.shape[0]
    L = [[Decimal(0)] * n for _ in range(n)]
    for j in range(n):
        s = Decimal(float(A[j, j])) - sum(L[j][p] * L[j][p] for p in range(j))
        L[j][j] = s.sqrt()
        for i in range(j + 1, n):
            t = Decimal(float(A[i, j])) - sum(L[i][p] * L[j][p] for p in range(j))
            L[i][j] = t / L[j][j]
    return np.array([[float(x) for x in row] for row in L])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_brute_force_tiny_50_digits(n):
    A = gen.spd_bbt(n, seed=100 + n)
    Lref = _decimal_cholesky(A)
    for transr, uplo in LAYOUTS:
        out, info = _pftrf(transr, uplo, A)
        assert info == 0
        L = _factor_full(transr, uplo, n, out)
        # cond(A) <= ~10 here: a few ulps of max |L| per entry
        assert np.max(np.abs(L - Lref)) <= 16 * n * EPS * np.max(np.abs(Lref))


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n,kind", [(33, "bbt"), (100, "spec"), (257, "bbt"), (256, "spec")])
def test_backward_error_bound(transr, uplo, n, kind):
    A = gen.spd_bbt(n, seed=n) if kind == "bbt" else gen.spd_spectrum(n, seed=n, kappa=1e4)
    out, info = _pftrf(transr, uplo, A)
    assert info == 0
    res = oracle.factor_residual(A, _factor_full(transr, uplo, n, out))
    assert res <= 64 * n * EPS and res <= 1e-13


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n,k", [(9, 0), (9, 3), (9, 5), (9, 8), (10, 4), (10, 5), (40, 30)])
def test_info_first_failing_minor(transr, uplo, n, k):
    A, L0 = gen.spd_integer_factor(n, seed=7)
    A = A.copy()
    A[k, k] -= L0[k, k] ** 2 + 1.0     # pivot k becomes exactly -1
    out, info = _pftrf(transr, uplo, A)
    assert info == k + 1


def test_info_nan_and_zero_pivot():
    A = np.eye(5)
    A[2, 2] = 0.0
    assert _pftrf("N", "L", A)[1] == 3
    A[2, 2] = np.nan
    assert _pftrf("T", "U", A)[1] == 3


# ---- solve ----------------------------------------------------------------

@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [1, 6, 13, 40])
def test_solve_integer_exact(transr, uplo, n):
    A, _ = gen.spd_integer_factor(n, seed=3 * n)
    X = np.asfortranarray(np.random.default_rng(n).integers(-3, 4, (n, 5)).astype(float))
    B = A @ X
    out, info = _pftrf(transr, uplo, A)
    assert info == 0
    np.testing.assert_array_equal(oracle.pftrs(transr, uplo, n, out, B), X)


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n,nrhs", [(1, 1), (64, 3), (101, 16), (200, 7)])
def test_solve_backward_error(transr, uplo, n, nrhs):
    A, rng = gen.spd_bbt(n, seed=n, return_rng=True)
    B = gen.rhs(n, nrhs, rng)
    out, _ = _pftrf(transr, uplo, A)
    X = oracle.pftrs(transr, uplo, n, out, B)
    assert oracle.solve_backward_error(A, X, B) <= 64 * n * EPS


# ---- inverse ----------------------------------------------------------------

@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [1, 2, 5, 16, 41])
def test_inverse_second_difference_closed_form(transr, uplo, n):
    K, Kinv = gen.second_difference(n)
    out, _ = _pftrf(transr, uplo, K)
    inv, info = oracle.pftri(transr, uplo, n, out)
    assert info == 0
    got = _sym_full(transr, uplo, n, inv)
    # cond(K) ~ 4 (n+1)^2 / pi^2; a forward error of a small multiple of cond * u
    cond = 4 * (n + 1) ** 2 / np.pi ** 2 + 1
    assert np.max(np.abs(got - Kinv)) <= 32 * cond * EPS * np.max(np.abs(Kinv))


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [3, 10, 24])
def test_inverse_integer_exact(transr, uplo, n):
    A, L0 = gen.spd_integer_factor(n, seed=11 * n, lo=-1, hi=1)
    W0 = np.round(np.linalg.inv(L0))           # integer: L0 is unit lower integer
    assert np.array_equal(L0 @ W0, np.eye(n))
    Ainv = W0.T @ W0
    out, _ = _pftrf(transr, uplo, A)
    inv, info = oracle.pftri(transr, uplo, n, out)
    assert info == 0
    np.testing.assert_array_equal(_sym_full(transr, uplo, n, inv), Ainv)


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n,kind", [(64, "bbt"), (129, "spec")])
def test_inverse_residual_bound(transr, uplo, n, kind):
    A = gen.spd_bbt(n, seed=n) if kind == "bbt" else gen.spd_spectrum(n, seed=n, kappa=1e4)
    out, _ = _pftrf(transr, uplo, A)
    inv, info = oracle.pftri(transr, uplo, n, out)
    assert info == 0
    assert oracle.inverse_residual(A, _sym_full(transr, uplo, n, inv)) <= 64 * n * EPS


def test_pftri_zero_diagonal_info():
    arf = oracle.pack("N", "L", np.diag([1.0, 2.0, 0.0, 4.0]))
    assert oracle.pftri("N", "L", 4, arf)[1] == 3


# ---- error measures -----------------------------------------------------------

def test_error_measures_on_known_cases():
    A, L0 = gen.spd_integer_factor(20, seed=1)
    assert oracle.factor_residual(A, L0) == 0.0
    L1 = L0.copy()
    L1[5, 2] += 1e-3
    r = oracle.factor_residual(A, L1)
    assert 1e-6 < r < 1e-2
    K, Kinv = gen.second_difference(12)
    assert oracle.inverse_residual(K, Kinv) < 1e-15
    X = np.ones((12, 1))
    assert oracle.solve_backward_error(K, X, K @ X) == 0.0
    assert oracle.solve_backward_error(K, X, K @ X + 1e-9) > 1e-11


# ---- external cross-check: LAPACK's RFP routines ------------------------------

@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [5, 64, 65, 300])
def test_matches_lapack_pftrf_pftrs_pftri(transr, uplo, n):
    la = pytest.importorskip("scipy.linalg.lapack")
    A, rng = gen.spd_bbt(n, seed=n, return_rng=True)
    B = gen.rhs(n, 4, rng)
    arf = oracle.pack(transr, uplo, A)
    ours, info = oracle.pftrf(transr, uplo, n, arf)
    ref, info2 = la.dpftrf(n, arf.copy(), transr=transr, uplo=uplo)
    assert info == info2 == 0
    assert np.max(np.abs(ours - ref)) <= 64 * n * EPS * np.max(np.abs(ref))
    X = oracle.pftrs(transr, uplo, n, ours, B)
    Xr, _ = la.dpftrs(n, ref, B.copy(order="F"), transr=transr, uplo=uplo)
    assert np.max(np.abs(X - Xr)) <= 64 * n * EPS * np.max(np.abs(Xr)) * 10
    inv, _ = oracle.pftri(transr, uplo, n, ours)
    invr, _ = la.dpftri(n, ref.copy(), transr=transr, uplo=uplo)
    assert np.max(np.abs(inv - invr)) <= 64 * n * EPS * np.max(np.abs(invr)) * 10
