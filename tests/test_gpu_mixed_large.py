"""The mixed-precision solve at n = 16384 for every precision and every
condition number of the mixed-precision configuration (kappa = 1e2, 1e4,
1e6), through the C ABI.

A = Q diag(lam) Q^T (random butterfly Q, lam log-uniform on [1, kappa] with
both ends pinned), packed by the oracle on the host.  Each solve must either
converge, with the device's backward error <= 1e-15 and the oracle's
compensated backward error <= 1e-14 on sampled columns, or report its
failure (a factorization breakdown in `info`, or converged = 0 after every
allowed step); it may never claim convergence it did not reach.  FP32 and
the two split modes (FP32-accurate updates on the tensor cores) must
converge at every kappa here: kappa * u_fp32 <= 6e-2.
"""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")

N, NRHS, MAX_ITER = 16384, 32, 30
PRECS = {"fp32": 2, "tf32x3": 3, "bf16x6": 4, "tf32": 1, "bf16": 0}
MUST_CONVERGE = {"fp32", "tf32x3", "bf16x6"}
SAMPLE = [0, NRHS // 2, NRHS - 1]


@pytest.fixture(scope="module", params=[1e2, 1e4, 1e6], ids=["k1e2", "k1e4", "k1e6"])
def system(request):
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    kappa = request.param
    A = gen.spd_butterfly(N, seed=0, kappa=kappa, device=torch.device("cuda")).cpu().numpy()
    B = gen.rhs(N, NRHS, seed=11)
    arf = torch.from_numpy(oracle.pack("N", "L", A)).cuda()
    yield kappa, A, B, arf
    del arf
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", list(PRECS))
def test_mixed_n16384_converges_or_reports(system, prec):
    kappa, A, B, arf = system
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    dX = torch.full((NRHS, N), np.nan, dtype=torch.float64, device="cuda")
    wb = rfp.rfp_dpfsv_mixed_workspace(N, NRHS, PRECS[prec])
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    status = torch.zeros(24, dtype=torch.uint8, device="cuda")
    rfp.rfp_dpfsv_mixed("N", "L", N, NRHS, arf, dB, N, dX, N, PRECS[prec], MAX_ITER, 1e-15, work,
                        wb, status)
    st = rfp.mixed_status(status.cpu().numpy().tobytes())
    assert st["tc_error"] == 0, st
    if prec in MUST_CONVERGE:
        assert st["info"] == 0 and st["converged"] == 1, (kappa, prec, st)
    if st["converged"] == 1:
        assert st["info"] == 0
        assert st["backward_error"] <= 1e-15
        X = dX.cpu().numpy().T
        assert oracle.solve_backward_error(A, X[:, SAMPLE], B[:, SAMPLE]) <= 1e-14, (kappa, prec)
    else:
        # an honest failure: a reported breakdown, or every step spent
        assert st["info"] > 0 or st["iterations"] == MAX_ITER, (kappa, prec, st)
    del work, dX
