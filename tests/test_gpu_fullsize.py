"""GPU parity at the benchmark's full size: n = 16384 and n = 16383, all
eight layouts, in the launch configuration bench.py times (pack, PFTRF,
PFTRS with nrhs = 256, PFTRI, unpack through the C ABI).

At this size the oracle cannot refactor the matrix, so the checks are
(a) bit-exact pack / unpack against the oracle's index maps,
(b) sampled outputs the oracle computes directly: the leading 384 x 384
    block of L is the Cholesky factor of A's leading block,
(c) properties that hold at any size, evaluated in FP64 on the CPU:
    the backward error of the factor estimated with 16 random probes,
    the normwise backward error of every solved column, and the inverse's
    residual on 16 random probes, each <= 1e-13.
"""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen
from rfp_inputs import LAYOUTS

from gpu_util import factor_tolerance

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")

NRHS = 256
LEAD = 384


@pytest.fixture(scope="module", params=[16384, 16383])
def problem(request):
    n = request.param
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    dA = gen.spd_spectrum(n, seed=0, kappa=1e4, device=torch.device("cuda"))
    A = dA.cpu().numpy()          # symmetric: row- and column-major agree
    Bh = gen.rhs(n, NRHS, seed=1)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((n, 16))
    lead_ref, info = oracle.potrf_full(A[:LEAD, :LEAD])
    assert info == 0
    yield dict(n=n, dA=dA, A=A, B=Bh, V=V, AV=A @ V, anorm=np.linalg.norm(A),
               lead=lead_ref)
    del dA
    torch.cuda.empty_cache()


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
def test_fullsize_path(problem, transr, uplo):
    n, dA, A, B = problem["n"], problem["dA"], problem["A"], problem["B"]
    nt = n * (n + 1) // 2
    arf = torch.empty(nt, dtype=torch.float64, device="cuda")
    info = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    X = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    rfp.rfp_dpack(transr, uplo, n, dA, n, arf)
    packed = arf.cpu().numpy()
    np.testing.assert_array_equal(packed, oracle.pack(transr, uplo, A))
    rfp.rfp_dpftrf(transr, uplo, n, arf, info[0:1])
    rfp.rfp_dpftrs(transr, uplo, n, NRHS, arf, X, n)
    fac = arf.cpu().numpy()
    Xh = np.asfortranarray(X.cpu().numpy().T)
    rfp.rfp_dpftri(transr, uplo, n, arf, info[1:2])
    Ainv = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    rfp.rfp_dunpack(transr, uplo, n, arf, Ainv, n)
    inv = arf.cpu().numpy()
    full_inv = Ainv.cpu().numpy().T
    assert info.cpu().tolist() == [0, 0]

    # unpack is the exact inverse map of pack
    np.testing.assert_array_equal(full_inv, oracle.unpack(transr, uplo, n, inv))

    F = oracle.unpack(transr, uplo, n, fac)
    L = np.tril(F) if uplo == "L" else np.triu(F).T
    del F
    # (b) sampled outputs: leading block
    lead = problem["lead"]
    assert np.max(np.abs(L[:LEAD, :LEAD] - lead)) <= factor_tolerance(n, 1e4) * np.max(np.abs(lead))
    # (c) backward error of the factor on random probes
    V = problem["V"]
    E = problem["AV"] - L @ (L.T @ V)
    est = np.sqrt(n) * np.linalg.norm(E) / (np.linalg.norm(V) * problem["anorm"])
    assert est <= 1e-13, est
    del L
    # solve: normwise backward error of every column
    R = B - A @ Xh
    anorm_inf = np.max(np.sum(np.abs(A), axis=1))
    bwd = np.max(np.max(np.abs(R), axis=0) /
                 (anorm_inf * np.max(np.abs(Xh), axis=0) + np.max(np.abs(B), axis=0)))
    assert bwd <= 1e-13, bwd
    # inverse: || A (Ainv V) - V || on probes
    S = np.tril(full_inv) + np.tril(full_inv, -1).T if uplo == "L" else \
        np.triu(full_inv) + np.triu(full_inv, 1).T
    res = np.linalg.norm(A @ (S @ V) - V) / (np.linalg.norm(V) * 1e4)   # kappa = 1e4
    assert res <= 1e-13 * np.sqrt(n), res
