"""GPU tests of the mixed-precision solve (rfp_dpfsv_mixed) through the C ABI.

The target: a normwise backward error max_j ||b_j - A x_j||_inf /
(||A||_inf ||x_j||_inf + ||b_j||_inf) <= 1e-14, checked both by the device's
own figure and independently by the oracle's compensated residual, and a
solution within the forward-error bound kappa * 1e-14 of the oracle's FP64
solve.  Refinement from a factor of unit roundoff u_f converges when
kappa * u_f < 1: FP32 up to kappa = 1e6, TF32 and BF16 only for small
kappa; where it cannot converge the status must say so (converged = 0 or a
reported factorization failure), never claim convergence.
"""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")

PRECS = {"fp32": 2, "tf32": 1, "bf16": 0, "tf32x3": 3, "bf16x6": 4}


def solve_mixed(transr, uplo, A, B, prec, max_iter=30, tol=1e-15):
    n, nrhs = B.shape
    arf = torch.from_numpy(oracle.pack(transr, uplo, A)).cuda()
    arf0 = arf.clone()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()          # column-major
    ldx = n + 1
    dX = torch.full((nrhs, ldx), np.nan, dtype=torch.float64, device="cuda")
    wb = rfp.rfp_dpfsv_mixed_workspace(n, nrhs, prec)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    status = torch.zeros(24, dtype=torch.uint8, device="cuda")
    rfp.rfp_dpfsv_mixed(transr, uplo, n, nrhs, arf, dB, n, dX, ldx, prec, max_iter, tol, work, wb,
                        status)
    st = rfp.mixed_status(status.cpu().numpy().tobytes())
    X = np.asfortranarray(dX.cpu().numpy()[:, :n].T)
    assert torch.equal(arf, arf0), "A must not be modified"
    return X, st


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x6", "tf32", "bf16"])
@pytest.mark.parametrize("transr,uplo,n", [("N", "L", 100), ("T", "U", 513), ("N", "U", 1300),
                                           ("T", "L", 2100)])
def test_mixed_converges_well_conditioned(prec, transr, uplo, n):
    A, rng = gen.spd_bbt(n, seed=n, return_rng=True)
    B = gen.rhs(n, 16, rng)
    X, st = solve_mixed(transr, uplo, A, B, PRECS[prec])
    assert st["info"] == 0 and st["tc_error"] == 0
    assert st["converged"] == 1, st
    assert st["backward_error"] <= 1e-15
    assert oracle.solve_backward_error(A, X, B) <= 1e-14
    ref = oracle.pftrs(transr, uplo, n, oracle.pftrf(transr, uplo, n, oracle.pack(transr, uplo, A))[0], B)
    assert np.max(np.abs(X - ref)) <= 10 * 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x6", "tf32", "bf16"])
def test_mixed_conditioning(prec, kappa):
    n = 1200
    A = gen.spd_spectrum(n, seed=7, kappa=kappa)
    B = gen.rhs(n, 8, seed=8)
    X, st = solve_mixed("N", "L", A, B, PRECS[prec], max_iter=40)
    assert st["tc_error"] == 0
    bwd = oracle.solve_backward_error(A, X, B) if st["info"] == 0 else np.inf
    u_f = {"fp32": 2.0 ** -24, "tf32x3": 2.0 ** -22, "bf16x6": 2.0 ** -22, "tf32": 2.0 ** -11,
           "bf16": 2.0 ** -8}[prec]
    if st["converged"]:
        assert st["backward_error"] <= 1e-15 and bwd <= 1e-14, (st, bwd)
    if kappa * u_f * 100 < 1:         # well inside the convergence condition
        assert st["info"] == 0 and st["converged"] == 1, st


def test_mixed_argument_checks():
    n, nrhs = 64, 2
    arf = torch.zeros(n * (n + 1) // 2, dtype=torch.float64, device="cuda")
    B = torch.zeros(nrhs, n, dtype=torch.float64, device="cuda")
    X = torch.zeros_like(B)
    wb = rfp.rfp_dpfsv_mixed_workspace(n, nrhs, 2)
    work = torch.empty(wb + 512, dtype=torch.uint8, device="cuda")
    status = torch.zeros(24, dtype=torch.uint8, device="cuda")
    bad = [((n, nrhs, arf, B, n, X, n, 7, 5, 1e-14, work, wb), -10),
           ((n, nrhs, arf, B, n - 1, X, n, 2, 5, 1e-14, work, wb), -7),
           ((n, nrhs, arf, B, n, X, n, 2, 5, 1e-14, work, wb - 8), -14),
           ((n, nrhs, arf, B, n, X, n, 2, 5, 1e-14, work.data_ptr() + 8, wb), -13),
           ((n, nrhs, arf, B, n, X, n, 2, -1, 1e-14, work, wb), -11)]
    for args, code in bad:
        with pytest.raises(rfp.RfpError) as e:
            rfp.rfp_dpfsv_mixed("N", "L", *args, status)
        assert e.value.status == code
    assert rfp.rfp_dpfsv_mixed_workspace(n, nrhs, 9) == 0


def test_tf32x3_refines_like_fp32():
    """The split-TF32 updates carry FP32's precision per operand: at kappa =
    1e4 the refinement needs at most two steps beyond the FP32 factor's and
    fewer than half of the plain TF32 factor's (measured on GB300: 3 / 5 /
    18 steps for FP32 / split-TF32 / TF32; the tensor cores' FP32
    accumulation is not the FMA pipe's)."""
    n = 2100
    A = gen.spd_spectrum(n, seed=11, kappa=1e4)
    B = gen.rhs(n, 8, seed=12)
    its = {}
    for name in ["fp32", "tf32x3", "tf32"]:
        _, st = solve_mixed("N", "L", A, B, PRECS[name], max_iter=40)
        assert st["info"] == 0 and st["converged"] == 1, (name, st)
        its[name] = st["iterations"]
    assert its["tf32x3"] <= its["fp32"] + 2 and 2 * its["tf32x3"] < its["tf32"], its


def test_bf16x6_reaches_fp64_accuracy_where_bf16_cannot():
    """kappa = 1e6: kappa u_bf16 >> 1, so the plain BF16 factor cannot drive
    the refinement; the split-BF16 updates (same tensor cores, six products)
    reach the FP64 bar like the FP32 factor."""
    n = 2100
    A = gen.spd_spectrum(n, seed=13, kappa=1e6)
    B = gen.rhs(n, 4, seed=14)
    X, st = solve_mixed("T", "L", A, B, PRECS["bf16x6"], max_iter=60)
    assert st["info"] == 0 and st["tc_error"] == 0 and st["converged"] == 1, st
    assert oracle.solve_backward_error(A, X, B) <= 1e-14
    _, st16 = solve_mixed("T", "L", A, B, PRECS["bf16"], max_iter=60)
    assert st16["info"] != 0 or st16["converged"] == 0


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "tf32"])
def test_mixed_large_split_k_residual(prec):
    """n = 8200: the refinement's FP64 residual products run split along K
    (two chunks) through the workspace; the solve must still meet the bar."""
    n = 8200
    A = gen.spd_bbt(n, seed=5)
    B = gen.rhs(n, 4, seed=6)
    X, st = solve_mixed("T", "U", A, B, PRECS[prec])
    assert st["info"] == 0 and st["tc_error"] == 0 and st["converged"] == 1, st
    assert oracle.solve_backward_error(A, X, B) <= 1e-14


@pytest.mark.parametrize("transr,uplo,n,nrhs", [("N", "L", 1000, 20), ("T", "U", 4097, 64),
                                                ("N", "U", 129, 1)])
def test_one_step_is_one_fp32_solve(transr, uplo, n, nrhs):
    """max_iter = 1: X = (L L^T)^{-1} fl32(B) with the FP32 factor, i.e. the
    one-launch block solves alone, against the oracle's FP64 solve (forward
    error of an FP32 solve of a well-conditioned system)."""
    A, rng = gen.spd_bbt(n, seed=n + 3, return_rng=True)
    B = gen.rhs(n, nrhs, rng)
    X, st = solve_mixed(transr, uplo, A, B, PRECS["fp32"], max_iter=1)
    assert st["info"] == 0 and st["tc_error"] == 0 and st["iterations"] == 1, st
    ref = oracle.pftrs(transr, uplo, n, oracle.pftrf(transr, uplo, n, oracle.pack(transr, uplo, A))[0], B)
    assert np.max(np.abs(X - ref)) <= 1e-4 * np.max(np.abs(ref))
