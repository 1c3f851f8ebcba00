"""GPU parity of the one-launch FP64 PFTRS (Section 4's block substitutions as
one launch per direction over the whole factor) against the oracle.

Covered here beyond test_gpu_parity.py: many right-hand sides with a ragged
last column group, orders whose T1 / T2 blocks end mid-tile on either side of
the n1 split, ldb > n with the rows beyond n left untouched, the multi-launch
form that runs under CUDA graph capture (it must agree with the one-launch
form within rounding and with the oracle), and two solves running at once
on two streams (each takes its own scratch: results equal to the same
solves run alone, bit for bit).
"""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen
from rfp_inputs import LAYOUTS

from gpu_util import dev_colmajor, factor_tolerance, host_colmajor

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    rfp.library()
    yield
    torch.cuda.synchronize()


def _factor(transr, uplo, A):
    n = A.shape[0]
    ref_f, info = oracle.pftrf(transr, uplo, n, oracle.pack(transr, uplo, A))
    assert info == 0
    return ref_f


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n,nrhs", [(1, 3), (2, 17), (65, 1), (129, 33), (700, 257), (1001, 16),
                                    (1103, 48)])
def test_one_launch_solve_vs_oracle(transr, uplo, n, nrhs):
    A, rng = gen.spd_bbt(n, seed=n + nrhs, return_rng=True)
    B = gen.rhs(n, nrhs, rng)
    ref_f = _factor(transr, uplo, A)
    arf = torch.from_numpy(ref_f).cuda()
    ldb = n + 5
    dB = dev_colmajor(torch, B, ld=ldb, fill=-7.0)
    rfp.rfp_dpftrs(transr, uplo, n, nrhs, arf, dB, ldb)
    X = host_colmajor(dB, n, nrhs)
    ref_x = oracle.pftrs(transr, uplo, n, ref_f, B)
    assert np.max(np.abs(X - ref_x)) <= factor_tolerance(n) * np.max(np.abs(ref_x))
    assert oracle.solve_backward_error(A, X, B) <= 1e-13
    assert np.all(dB.cpu().numpy()[:nrhs, n:] == -7.0)          # rows beyond n untouched
    assert np.array_equal(arf.cpu().numpy(), ref_f)              # the factor is read only


@pytest.mark.parametrize("transr,uplo", [("N", "L"), ("T", "U")])
def test_captured_solve_matches_direct_solve(transr, uplo):
    n, nrhs = 611, 40
    A, rng = gen.spd_spectrum(n, seed=5, kappa=1e4), np.random.default_rng(3)
    B = gen.rhs(n, nrhs, rng)
    ref_f = _factor(transr, uplo, A)
    arf = torch.from_numpy(ref_f).cuda()
    d_direct = dev_colmajor(torch, B)
    rfp.rfp_dpftrs(transr, uplo, n, nrhs, arf, d_direct, n)
    B0 = dev_colmajor(torch, B)
    d_graph = B0.clone()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rfp.rfp_dpftrs(transr, uplo, n, nrhs, arf, d_graph, n, stream=s)
    for _ in range(2):                      # replay twice on fresh inputs
        d_graph.copy_(B0)
        g.replay()
    torch.cuda.synchronize()
    X1 = host_colmajor(d_direct, n, nrhs)
    X2 = host_colmajor(d_graph, n, nrhs)
    ref_x = oracle.pftrs(transr, uplo, n, ref_f, B)
    tol = factor_tolerance(n, kappa=1e4) * np.max(np.abs(ref_x))
    assert np.max(np.abs(X1 - ref_x)) <= tol
    assert np.max(np.abs(X2 - ref_x)) <= tol
    assert np.max(np.abs(X1 - X2)) <= tol
    assert oracle.solve_backward_error(A, X2, B) <= 1e-13


def test_two_streams_at_once_equal_alone():
    cases = [("N", "L", 1500, 64, 1), ("T", "U", 1201, 33, 2)]
    inputs, alone = [], []
    for transr, uplo, n, nrhs, seed in cases:
        A, rng = gen.spd_bbt(n, seed=seed, return_rng=True)
        B = gen.rhs(n, nrhs, rng)
        arf = torch.from_numpy(_factor(transr, uplo, A)).cuda()
        d = dev_colmajor(torch, B)
        rfp.rfp_dpftrs(transr, uplo, n, nrhs, arf, d, n)
        alone.append(host_colmajor(d, n, nrhs))
        inputs.append((transr, uplo, n, nrhs, arf, dev_colmajor(torch, B), A, B))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    for rep in range(3):
        outs = [x[5].clone() for x in inputs]
        torch.cuda.synchronize()
        for (transr, uplo, n, nrhs, arf, _, _, _), d, s in zip(inputs, outs, streams):
            rfp.rfp_dpftrs(transr, uplo, n, nrhs, arf, d, n, stream=s)
        torch.cuda.synchronize()
        for (transr, uplo, n, nrhs, _, _, A, B), d, ref in zip(inputs, outs, alone):
            X = host_colmajor(d, n, nrhs)
            assert np.array_equal(X, ref)
            assert oracle.solve_backward_error(A, X, B) <= 1e-13


@pytest.mark.parametrize("transr,uplo,n", [("N", "L", 700), ("T", "U", 385), ("N", "U", 1001)])
def test_captured_factor_solve_inverse_match_direct(transr, uplo, n):
    """Under CUDA graph capture PFTRF, PFTRS and PFTRI run their
    multi-launch forms (no scratch is taken while capturing); replayed, they
    must agree with the direct calls (lookahead steps and one-launch solves)
    within rounding, and with the oracle."""
    nrhs = 20
    A, rng = gen.spd_bbt(n, seed=n + 3, return_rng=True)
    B = gen.rhs(n, nrhs, rng)
    arf0 = torch.from_numpy(oracle.pack(transr, uplo, A)).cuda()
    B0 = dev_colmajor(torch, B)
    info = torch.zeros(2, dtype=torch.int32, device="cuda")

    def run(arf, dB, stream=None):
        rfp.rfp_dpftrf(transr, uplo, n, arf, info[0:1], stream=stream)
        rfp.rfp_dpftrs(transr, uplo, n, nrhs, arf, dB, n, stream=stream)
        fac = arf.clone()
        rfp.rfp_dpftri(transr, uplo, n, arf, info[1:2], stream=stream)
        return fac

    a1, b1 = arf0.clone(), B0.clone()
    f1 = run(a1, b1)
    torch.cuda.synchronize()
    assert int(info.abs().sum().item()) == 0
    a2, b2 = arf0.clone(), B0.clone()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        f2 = run(a2, b2, stream=s)
    a2.copy_(arf0)
    b2.copy_(B0)
    info.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert int(info.abs().sum().item()) == 0
    ref_f, _ = oracle.pftrf(transr, uplo, n, oracle.pack(transr, uplo, A))
    ref_x = oracle.pftrs(transr, uplo, n, ref_f, B)
    ref_i, _ = oracle.pftri(transr, uplo, n, ref_f)
    tol = factor_tolerance(n)
    for got, ref in ((f1, ref_f), (f2, ref_f), (a1, ref_i), (a2, ref_i)):
        got = got.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    for dB in (b1, b2):
        X = host_colmajor(dB, n, nrhs)
        assert np.max(np.abs(X - ref_x)) <= tol * np.max(np.abs(ref_x))
        assert oracle.solve_backward_error(A, X, B) <= 1e-13
