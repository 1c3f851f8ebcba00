"""GPU test of the tcgen05 tensor-core SYRK (rfp_ssyrk_tc) against an FP64
product of the same low-precision inputs, computed on the CPU.

BF16 inputs: every product of two BF16 values is exact in FP32, so the only
error is the FP32 accumulation: |C - C_ref| <= k * 2^-23 * sum |a_ip a_jp|
(with headroom).  TF32 inputs: the tensor core reads the FP32 operands at
TF32 precision (10-bit mantissa), which adds up to 2 * 2^-10 of the same
sum.  The strict upper triangle of C must be untouched and the kernel's
error flag must stay 0.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")


def _case(n, k, prec, alpha=-1.0, beta=1.0, seed=0):
    g = torch.Generator().manual_seed(seed)
    A32 = (torch.rand(n, k, generator=g, dtype=torch.float32) * 2 - 1)
    esz = 2 if prec == rfp.RFP_PREC_BF16 else 4
    lda = ((k + 16 // esz - 1) // (16 // esz)) * (16 // esz) + (16 // esz)   # padded, aligned pitch
    if prec == rfp.RFP_PREC_BF16:
        Aq = A32.to(torch.bfloat16)
        buf = torch.zeros(n, lda, dtype=torch.bfloat16)
        buf[:, :k] = Aq
        Aref = Aq.to(torch.float64).numpy()
    else:
        buf = torch.zeros(n, lda, dtype=torch.float32)
        buf[:, :k] = A32
        Aref = A32.to(torch.float64).numpy()
    C0 = torch.rand(n, n, generator=g, dtype=torch.float32)          # row-major (n, n) = C^T
    dA, dC = buf.cuda(), C0.clone().cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rfp.rfp_ssyrk_tc("L", n, k, alpha, dA, lda, prec, beta, dC, n, err)
    C = dC.cpu().numpy().T.astype(np.float64)                        # column-major view
    Cin = C0.numpy().T.astype(np.float64)
    ref = alpha * (Aref @ Aref.T) + beta * Cin
    mag = np.abs(Aref) @ np.abs(Aref).T
    return C, Cin, ref, mag, int(err.item())


@pytest.mark.parametrize("n,k", [(128, 64), (200, 100), (256, 128), (129, 1), (1000, 300),
                                 (384, 1024), (1, 64)])
def test_tc_syrk_bf16(n, k):
    C, Cin, ref, mag, err = _case(n, k, rfp.RFP_PREC_BF16)
    assert err == 0
    low = np.tril(np.ones((n, n), bool))
    tol = 4 * k * 2.0 ** -23 * mag + 4 * 2.0 ** -23 * np.abs(ref)
    bad = np.abs(C - ref) > tol
    assert not np.any(bad & low), np.max(np.abs(C - ref)[low])
    np.testing.assert_array_equal(C[~low], Cin[~low])


@pytest.mark.parametrize("n,k", [(128, 32), (300, 200), (512, 512)])
def test_tc_syrk_tf32(n, k):
    C, Cin, ref, mag, err = _case(n, k, rfp.RFP_PREC_TF32)
    assert err == 0
    low = np.tril(np.ones((n, n), bool))
    tol = (4 * 2.0 ** -10 + 4 * k * 2.0 ** -23) * mag + 4 * 2.0 ** -23 * np.abs(ref)
    assert not np.any((np.abs(C - ref) > tol) & low), np.max(np.abs(C - ref)[low])
    np.testing.assert_array_equal(C[~low], Cin[~low])


@pytest.mark.parametrize("n,k,prec", [(4000, 96, 0), (2600, 64, 1), (3001, 200, 0)])
def test_tc_syrk_several_tiles_per_cta(n, k, prec):
    """More lower-triangular 128 x 128 tiles than SMs: every CTA of the
    persistent kernel walks several tiles, alternating its two accumulators
    (their barriers go through several phases), with ragged edge tiles."""
    p = rfp.RFP_PREC_BF16 if prec == 0 else rfp.RFP_PREC_TF32
    C, Cin, ref, mag, err = _case(n, k, p, seed=n)
    assert err == 0
    low = np.tril(np.ones((n, n), bool))
    rel = 4 * 2.0 ** -10 if p == rfp.RFP_PREC_TF32 else 0.0
    tol = (rel + 4 * k * 2.0 ** -23) * mag + 4 * 2.0 ** -23 * np.abs(ref)
    assert not np.any((np.abs(C - ref) > tol) & low), np.max(np.abs(C - ref)[low])
    np.testing.assert_array_equal(C[~low], Cin[~low])


def test_tc_syrk_beta_zero_ignores_c():
    n, k = 160, 96
    g = torch.Generator().manual_seed(3)
    A = (torch.rand(n, k, generator=g) * 2 - 1).to(torch.bfloat16)
    dA = A.cuda()
    dC = torch.full((n, n), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rfp.rfp_ssyrk_tc("L", n, k, 1.0, dA, k, rfp.RFP_PREC_BF16, 0.0, dC, n, err)
    C = dC.cpu().numpy().T
    low = np.tril(np.ones((n, n), bool))
    Ar = A.to(torch.float64).numpy()
    assert np.all(np.isfinite(C[low]))
    assert np.max(np.abs(C[low] - (Ar @ Ar.T)[low])) <= 4 * k * 2.0 ** -23 * np.max(np.abs(Ar) @ np.abs(Ar).T)
    assert int(err.item()) == 0


def test_tc_syrk_argument_checks():
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    A = torch.zeros(64, 24, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(64, 64, device="cuda")
    cases = [(("U", 64, 24, 1.0, A, 24, 0, 0.0, C, 64, err), -1),
             (("L", 64, 24, 1.0, A, 20, 0, 0.0, C, 64, err), -6),     # lda < k
             (("L", 64, 20, 1.0, A, 21, 0, 0.0, C, 64, err), -6),     # pitch not 16 B
             (("L", 64, 24, 1.0, A, 24, 5, 0.0, C, 64, err), -7),
             (("L", 64, 24, 1.0, A, 24, 0, 0.0, C, 63, err), -10)]
    for args, code in cases:
        with pytest.raises(rfp.RfpError) as e:
            rfp.rfp_ssyrk_tc(*args)
        assert e.value.status == code
