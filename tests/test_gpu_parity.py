"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Index work (pack / unpack) must be bit-exact.  Floating-point results are
compared element by element with the oracle within the forward-error
tolerance of two backward-stable Cholesky computations (gpu_util.
factor_tolerance), and the GPU result's own backward error must be at most
1e-13, the bound the FP64 path is held to.  Closed-form inputs whose every
intermediate is an integer (Pascal, integer factors) must be reproduced
exactly.  Sizes span one tile, several 64-wide tiles with ragged tails, and
the n = 1001 workload; the n = 16384 / 16383 workloads are in
test_gpu_fullsize.py.
"""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen
from rfp_inputs import LAYOUTS

from gpu_util import EPS32, EPS64, dev_colmajor, factor_tolerance, host_colmajor

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")

SMALL = [1, 2, 3, 5, 8, 17, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 192, 193, 257, 513]


def _arf(values, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(values)).to(dtype).cuda()


def _info():
    return torch.full((1,), -99, dtype=torch.int32, device="cuda")


def _lower(transr, uplo, n, arf_host):
    F = oracle.unpack(transr, uplo, n, arf_host)
    return np.tril(F) if uplo == "L" else np.triu(F).T


def _sym(transr, uplo, n, arf_host):
    F = oracle.unpack(transr, uplo, n, arf_host)
    return np.tril(F) + np.tril(F, -1).T if uplo == "L" else np.triu(F) + np.triu(F, 1).T


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    rfp.library()     # fail loudly if the CUDA library was not built
    yield
    torch.cuda.synchronize()


# ---- pack / unpack: bit-exact ----------------------------------------------------

@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 7, 8, 31, 63, 64, 65, 127, 128, 129, 256, 257, 1000, 1001])
@pytest.mark.parametrize("prec", ["d", "s"])
def test_pack_unpack_bit_exact(transr, uplo, n, prec):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    if prec == "s":
        A = A.astype(np.float32).astype(np.float64)
    dt = torch.float64 if prec == "d" else torch.float32
    lda = n + 5
    dA = dev_colmajor(torch, A, ld=lda, dtype=dt)
    arf = torch.full((max(n * (n + 1) // 2, 1),), np.nan, dtype=dt, device="cuda")
    getattr(rfp, f"rfp_{prec}pack")(transr, uplo, n, dA, lda, arf)
    got = arf.cpu().numpy().astype(np.float64)[: n * (n + 1) // 2]
    np.testing.assert_array_equal(got, oracle.pack(transr, uplo, A))
    # unpack into a sentinel-filled matrix: the other triangle and the rows
    # beyond n stay untouched
    out = dev_colmajor(torch, np.zeros((n, n)), ld=lda, dtype=dt, fill=-3.0)
    if n:
        out[:, :n] = -3.0
    getattr(rfp, f"rfp_{prec}unpack")(transr, uplo, n, arf, out, lda)
    full = out.cpu().numpy().astype(np.float64)
    back = full[:n, :n].T if n else np.zeros((0, 0))
    np.testing.assert_array_equal(back, oracle.unpack(transr, uplo, n, oracle.pack(transr, uplo, A),
                                                      np.full((n, n), -3.0)))
    assert np.all(full[:n, n:] == -3.0)


# ---- PFTRF / PFTRS / PFTRI against the oracle -------------------------------------

def _run_all(transr, uplo, A, B, nrhs):
    n = A.shape[0]
    arf = _arf(oracle.pack(transr, uplo, A))
    info = _info()
    rfp.rfp_dpftrf(transr, uplo, n, arf, info)
    fac = arf.cpu().numpy()
    info_f = int(info.item())
    ldb = n + 3
    dB = dev_colmajor(torch, B, ld=ldb)
    rfp.rfp_dpftrs(transr, uplo, n, nrhs, arf, dB, ldb)
    X = host_colmajor(dB, n, nrhs)
    rfp.rfp_dpftri(transr, uplo, n, arf, info)
    inv = arf.cpu().numpy()
    return fac, info_f, X, inv, int(info.item())


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", SMALL + [1001])
def test_factor_solve_inverse_vs_oracle(transr, uplo, n):
    nrhs = 16 if n % 2 else 70
    A, rng = gen.spd_bbt(n, seed=n, return_rng=True)
    B = gen.rhs(n, nrhs, rng)
    fac, info_f, X, inv, info_i = _run_all(transr, uplo, A, B, nrhs)
    assert info_f == 0 and info_i == 0

    ref_f, _ = oracle.pftrf(transr, uplo, n, oracle.pack(transr, uplo, A))
    tol = factor_tolerance(n)
    assert np.max(np.abs(fac - ref_f)) <= tol * np.max(np.abs(ref_f))
    assert oracle.factor_residual(A, _lower(transr, uplo, n, fac)) <= 1e-13

    ref_x = oracle.pftrs(transr, uplo, n, ref_f, B)
    assert np.max(np.abs(X - ref_x)) <= tol * np.max(np.abs(ref_x))
    assert oracle.solve_backward_error(A, X, B) <= 1e-13

    ref_i, _ = oracle.pftri(transr, uplo, n, ref_f)
    assert np.max(np.abs(inv - ref_i)) <= tol * np.max(np.abs(ref_i))
    assert oracle.inverse_residual(A, _sym(transr, uplo, n, inv)) <= 1e-13


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [130, 385])
def test_ill_conditioned_kappa_1e4(transr, uplo, n):
    A, rng = gen.spd_spectrum(n, seed=n, kappa=1e4), np.random.default_rng(1)
    B = gen.rhs(n, 8, rng)
    fac, info_f, X, inv, info_i = _run_all(transr, uplo, A, B, 8)
    assert info_f == 0 and info_i == 0
    ref_f, _ = oracle.pftrf(transr, uplo, n, oracle.pack(transr, uplo, A))
    assert np.max(np.abs(fac - ref_f)) <= factor_tolerance(n, 1e4) * np.max(np.abs(ref_f))
    assert oracle.factor_residual(A, _lower(transr, uplo, n, fac)) <= 1e-13
    assert oracle.solve_backward_error(A, X, B) <= 1e-13
    assert oracle.inverse_residual(A, _sym(transr, uplo, n, inv)) <= 1e-13


# ---- exact closed forms --------------------------------------------------------------

@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [5, 19])
def test_pascal_exact(transr, uplo, n):
    P, Lx = gen.pascal(n)
    arf = _arf(oracle.pack(transr, uplo, P))
    info = _info()
    rfp.rfp_dpftrf(transr, uplo, n, arf, info)
    assert int(info.item()) == 0
    np.testing.assert_array_equal(_lower(transr, uplo, n, arf.cpu().numpy()), Lx)


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [64, 100, 130, 200])
def test_integer_factor_solve_inverse_exact(transr, uplo, n):
    A, L0 = gen.spd_integer_factor(n, seed=n, lo=-1, hi=1)
    X0 = np.random.default_rng(n).integers(-3, 4, (n, 3)).astype(float)
    B = A @ X0
    fac, info_f, X, inv, info_i = _run_all(transr, uplo, A, B, 3)
    assert info_f == 0 and info_i == 0
    np.testing.assert_array_equal(_lower(transr, uplo, n, fac), L0)
    np.testing.assert_array_equal(X, X0)
    W0 = np.round(np.linalg.inv(L0))
    if np.max(np.abs(W0.T @ W0)) < 2.0 ** 50:       # integer inverse, exactly representable
        np.testing.assert_array_equal(_sym(transr, uplo, n, inv), W0.T @ W0)


# ---- failure reporting ------------------------------------------------------------------

@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n,k", [(9, 0), (9, 4), (9, 8), (200, 30), (200, 99), (200, 100),
                                 (200, 150), (200, 199)])
def test_info_first_failing_minor(transr, uplo, n, k):
    A, L0 = gen.spd_integer_factor(n, seed=2)
    A = A.copy()
    A[k, k] -= L0[k, k] ** 2 + 1.0
    arf = _arf(oracle.pack(transr, uplo, A))
    info = _info()
    rfp.rfp_dpftrf(transr, uplo, n, arf, info)
    assert int(info.item()) == k + 1 == oracle.pftrf(transr, uplo, n, oracle.pack(transr, uplo, A))[1]


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
def test_pftri_zero_diagonal_info(transr, uplo):
    n = 150
    d = np.ones(n)
    d[97] = 0.0
    arf = _arf(oracle.pack(transr, uplo, np.diag(d)))
    info = _info()
    rfp.rfp_dpftri(transr, uplo, n, arf, info)
    assert int(info.item()) == 98


def test_n_zero_sets_info_zero():
    info = _info()
    rfp.rfp_dpftrf("N", "L", 0, 0, info)
    assert int(info.item()) == 0


# ---- single precision ---------------------------------------------------------------------

@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [33, 200, 1001])
def test_single_precision(transr, uplo, n):
    A, rng = gen.spd_bbt(n, seed=n, return_rng=True)
    A32 = A.astype(np.float32).astype(np.float64)
    B = gen.rhs(n, 8, rng).astype(np.float32).astype(np.float64)
    arf = _arf(oracle.pack(transr, uplo, A32), torch.float32)
    info = _info()
    rfp.rfp_spftrf(transr, uplo, n, arf, info)
    assert int(info.item()) == 0
    fac = arf.cpu().numpy().astype(np.float64)
    ref_f, _ = oracle.pftrf(transr, uplo, n, oracle.pack(transr, uplo, A32))
    assert np.max(np.abs(fac - ref_f)) <= factor_tolerance(n, eps=EPS32) * np.max(np.abs(ref_f))
    assert oracle.factor_residual(A32, _lower(transr, uplo, n, fac)) <= 64 * n * EPS32
    dB = dev_colmajor(torch, B, dtype=torch.float32)
    rfp.rfp_spftrs(transr, uplo, n, 8, arf, dB, n)
    X = host_colmajor(dB, n, 8)
    assert oracle.solve_backward_error(A32, X, B) <= 64 * n * EPS32
    rfp.rfp_spftri(transr, uplo, n, arf, info)
    assert int(info.item()) == 0
    inv = arf.cpu().numpy().astype(np.float64)
    assert oracle.inverse_residual(A32, _sym(transr, uplo, n, inv)) <= 64 * n * EPS32


# ---- stream semantics -------------------------------------------------------------------------

def test_runs_on_the_given_stream():
    n = 300
    A, rng = gen.spd_bbt(n, seed=9, return_rng=True)
    s = torch.cuda.Stream()
    arf = _arf(oracle.pack("N", "L", A))
    info = _info()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        rfp.rfp_dpftrf("N", "L", n, arf, info, stream=s)
    s.synchronize()
    ref, _ = oracle.pftrf("N", "L", n, oracle.pack("N", "L", A))
    assert np.max(np.abs(arf.cpu().numpy() - ref)) <= factor_tolerance(n) * np.max(np.abs(ref))


@pytest.mark.parametrize("transr,uplo", [("N", "L"), ("T", "U"), ("N", "U"), ("T", "L")])
def test_pftrf_diagonal_pivots_within_ulps(transr, uplo):
    """The FP64 pivots' square roots come from a Newton-Raphson reciprocal
    square root (about a few ulp); for a diagonal A, L = diag(sqrt(a_ii)) must
    be within 4 ulp of the correctly rounded square root (numpy's, IEEE) over
    the whole normal exponent range, subnormal entries included (they take
    the exact path), with every off-diagonal entry exactly zero.  n = 300
    spans the first panel (tile POTRF) and the lookahead steps."""
    n = 300
    rng = np.random.default_rng(5)
    d = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-1020, 1020, n))
    d[:12] = [1.0, 2.0, 4.0, 0.25, 3.0, 1e-300, 1e300, 1.7e308, 2.3e-308, 1e-310, 5e-324, 0.5]
    A = np.diag(d)
    arf = _arf(oracle.pack(transr, uplo, A))
    info = _info()
    rfp.rfp_dpftrf(transr, uplo, n, arf, info)
    assert int(info.item()) == 0
    L = _lower(transr, uplo, n, arf.cpu().numpy())
    ref = np.sqrt(d)
    assert np.all(np.abs(np.diag(L) - ref) <= 4 * np.spacing(ref))
    assert np.count_nonzero(L - np.diag(np.diag(L))) == 0
