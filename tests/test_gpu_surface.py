"""GPU parity of the rest of the LAPACK 3.2 RFP routine set (TPTTF / TFTTP,
TFTRI, SFRK, TFSM, LANSF) through the C ABI against the oracle: bit-exact
for the format conversions, within the rounding bound for the arithmetic."""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen

from gpu_util import EPS32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")

LAYOUTS = [(t, u) for t in "NT" for u in "LU"]
SIZES = [1, 2, 63, 64, 65, 129, 1001, 2049]
f64 = torch.float64


def dev(x, dtype=f64):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def tri_arf(transr, uplo, n, seed):
    L = np.linalg.cholesky(gen.spd_bbt(n, seed=seed))
    return oracle.pack(transr, uplo, L if uplo == "L" else L.T)


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", SIZES)
def test_tpttf_tfttp_bit_exact(transr, uplo, n):
    ap = np.random.default_rng(n).standard_normal(n * (n + 1) // 2)
    d_ap, d_arf = dev(ap), torch.empty(ap.size, dtype=f64, device="cuda")
    rfp.rfp_dtpttf(transr, uplo, n, d_ap, d_arf)
    assert np.array_equal(d_arf.cpu().numpy(), oracle.tpttf(transr, uplo, n, ap))
    back = torch.empty_like(d_ap)
    rfp.rfp_dtfttp(transr, uplo, n, d_arf, back)
    assert torch.equal(back, d_ap)
    s_arf = torch.empty(ap.size, dtype=torch.float32, device="cuda")
    rfp.rfp_stpttf(transr, uplo, n, d_ap.float(), s_arf)
    assert np.array_equal(s_arf.cpu().numpy(), oracle.tpttf(transr, uplo, n, ap).astype(np.float32))


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [1, 65, 1001, 2049])
@pytest.mark.parametrize("diag", "NU")
def test_tftri(transr, uplo, n, diag):
    tri = tri_arf(transr, uplo, n, seed=n)
    ref, info_ref = oracle.tftri(transr, uplo, diag, n, tri)
    d = dev(tri)
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    work = torch.empty(n, dtype=f64, device="cuda")
    rfp.rfp_dtftri(transr, uplo, diag, n, d, info, work)
    assert int(info.item()) == info_ref == 0
    assert np.max(np.abs(d.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    if diag == "U":   # the stored diagonal comes back unchanged
        got = oracle.unpack(transr, uplo, n, d.cpu().numpy())
        assert np.array_equal(np.diag(got), np.diag(oracle.unpack(transr, uplo, n, tri)))


def test_tftri_zero_diagonal_info():
    n = 300
    L = np.tril(np.ones((n, n))) + np.eye(n)
    L[150, 150] = 0.0
    d = dev(oracle.pack("T", "L", L))
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    rfp.rfp_dtftri("T", "L", "N", n, d, info)
    assert int(info.item()) == 151


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n,k", [(1, 1), (65, 3), (1001, 130), (2049, 64), (300, 0)])
@pytest.mark.parametrize("trans", "NT")
def test_sfrk(transr, uplo, n, k, trans):
    rng = np.random.default_rng(n + k)
    A = rng.standard_normal((n, k) if trans == "N" else (k, n))
    C = rng.standard_normal((n, n))
    arf = oracle.pack(transr, uplo, C + C.T)
    for alpha, beta in ((0.75, -1.5), (1.0, 0.0), (0.0, 2.0)):
        ref = oracle.sfrk(transr, uplo, trans, n, k, alpha, A, beta, arf)
        d = dev(arf)
        dA = torch.from_numpy(np.asfortranarray(A).T.copy()).cuda() if A.size else \
            torch.zeros(1, dtype=f64, device="cuda")   # column-major A
        rfp.rfp_dsfrk(transr, uplo, trans, n, k, alpha, dA, max(1, A.shape[0]), beta, d)
        scale = max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(d.cpu().numpy() - ref)) <= 1e-13 * max(k, 1) * scale


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("side", "LR")
@pytest.mark.parametrize("trans", "NT")
@pytest.mark.parametrize("diag", "NU")
def test_tfsm(transr, uplo, side, trans, diag):
    for order, other in ((65, 7), (1001, 33)):
        tri = tri_arf(transr, uplo, order, seed=order + 5)
        m, nc = (order, other) if side == "L" else (other, order)
        B = np.random.default_rng(order).standard_normal((m, nc))
        ref = oracle.tfsm(transr, side, uplo, trans, diag, m, nc, -0.5, tri, B)
        ldb = m + 3
        Bw = np.zeros((ldb, nc), order="F")
        Bw[:m] = B
        dB = torch.from_numpy(Bw.T.copy()).cuda()          # column-major, ld = ldb
        rfp.rfp_dtfsm(transr, side, uplo, trans, diag, m, nc, -0.5, dev(tri), dB, ldb)
        got = dB.cpu().numpy().T[:m]
        assert np.max(np.abs(got - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))
        assert np.array_equal(dB.cpu().numpy().T[m:], np.zeros((ldb - m, nc)))   # ldb padding untouched


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [1, 64, 1001, 2049])
def test_lansf(transr, uplo, n):
    S = np.random.default_rng(n).standard_normal((n, n))
    arf = oracle.pack(transr, uplo, S + S.T)
    d = dev(arf)
    work = torch.empty(2 * n, dtype=f64, device="cuda")
    val = torch.empty(1, dtype=f64, device="cuda")
    for norm in "M1OIFE":
        rfp.rfp_dlansf(norm, transr, uplo, n, d, work, val)
        ref = oracle.lansf(norm, transr, uplo, n, arf)
        assert abs(val.item() - ref) <= 1e-13 * ref, norm
    # FP32, and a NaN entry propagates
    w32 = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    v32 = torch.empty(1, dtype=torch.float32, device="cuda")
    rfp.rfp_slansf("F", transr, uplo, n, d.float(), w32, v32)
    assert abs(v32.item() - oracle.lansf("F", transr, uplo, n, arf)) <= 1e-5 * v32.item()
    d[n // 2] = float("nan")
    rfp.rfp_dlansf("M", transr, uplo, n, d, work, val)
    assert np.isnan(val.item())


def test_single_precision_solve_and_update():
    n, transr, uplo = 777, "N", "U"
    tri = tri_arf(transr, uplo, n, seed=9)
    B = np.random.default_rng(9).standard_normal((n, 5))
    ref = oracle.tfsm(transr, "L", uplo, "T", "N", n, 5, 1.0, tri, B)
    dB = torch.from_numpy(B.T.copy()).cuda().float()
    rfp.rfp_stfsm(transr, "L", uplo, "T", "N", n, 5, 1.0, dev(tri, torch.float32), dB, n)
    assert np.max(np.abs(dB.cpu().numpy().T - ref)) <= 1e3 * EPS32 * np.max(np.abs(ref))
    A = np.random.default_rng(10).standard_normal((n, 40))
    C = oracle.pack(transr, uplo, np.eye(n))
    ref = oracle.sfrk(transr, uplo, "N", n, 40, 1.0, A, 1.0, C)
    dC = dev(C, torch.float32)
    rfp.rfp_ssfrk(transr, uplo, "N", n, 40, 1.0, torch.from_numpy(A.T.copy()).cuda().float(), n, 1.0, dC)
    assert np.max(np.abs(dC.cpu().numpy() - ref)) <= 100 * EPS32 * np.max(np.abs(ref))


def test_argument_checks():
    d = torch.zeros(10, dtype=f64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cases = [(lambda: rfp.rfp_dtftri("N", "L", "X", 4, d, info), -3),
             (lambda: rfp.rfp_dtftri("N", "L", "U", 4, d, info, None), -7),
             (lambda: rfp.rfp_dsfrk("N", "L", "Q", 4, 2, 1.0, d, 4, 0.0, d), -3),
             (lambda: rfp.rfp_dsfrk("N", "L", "N", 4, 2, 1.0, d, 3, 0.0, d), -8),
             (lambda: rfp.rfp_dtfsm("N", "X", "L", "N", "N", 4, 1, 1.0, d, d, 4), -2),
             (lambda: rfp.rfp_dtfsm("N", "L", "L", "N", "N", 4, 1, 1.0, d, d, 3), -11),
             (lambda: rfp.rfp_dlansf("Z", "N", "L", 4, d, d, d), -1),
             (lambda: rfp.rfp_dtpttf("C", "L", 4, d, d), -1)]
    for f, code in cases:
        with pytest.raises(rfp.RfpError) as e:
            f()
        assert e.value.status == code
