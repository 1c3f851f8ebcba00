"""GPU parity at the orders where the FP64 kernels change shape, element by
element against the oracle (which still factors and inverts these orders in
seconds):

* n = 4100: triangles of order 2050, i.e. lookahead steps with 32-wide
  panels and 64-row strips, one-launch solves with 64-row blocks;
* n = 6001: the same kernels at odd n (T1 one row longer than T2);
* n = 8200: triangles of order 4100, i.e. 64-wide panels with 64-row strips.

Each runs PFTRF, PFTRS (8-column and 16-column task groups) and PFTRI
through the C ABI.
"""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen

from gpu_util import dev_colmajor, factor_tolerance, host_colmajor

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")


@pytest.mark.parametrize("transr,uplo,n,nrhs", [("N", "L", 4100, 12), ("T", "U", 6001, 40),
                                                ("N", "U", 8200, 16)])
def test_midsize_factor_solve_inverse(transr, uplo, n, nrhs):
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    A = gen.spd_spectrum(n, seed=n, kappa=1e4, device=torch.device("cuda")).cpu().numpy()
    B = gen.rhs(n, nrhs, seed=n + 1)
    packed = oracle.pack(transr, uplo, A)
    ref_f, info = oracle.pftrf(transr, uplo, n, packed)
    assert info == 0
    arf = torch.from_numpy(packed).cuda()
    info_d = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    rfp.rfp_dpftrf(transr, uplo, n, arf, info_d[0:1])
    got_f = arf.cpu().numpy()
    tol = factor_tolerance(n, kappa=1e4)
    assert int(info_d[0].item()) == 0
    assert np.max(np.abs(got_f - ref_f)) <= tol * np.max(np.abs(ref_f))

    dB = dev_colmajor(torch, B)
    rfp.rfp_dpftrs(transr, uplo, n, nrhs, arf, dB, n)
    X = host_colmajor(dB, n, nrhs)
    ref_x = oracle.pftrs(transr, uplo, n, ref_f, B)
    assert np.max(np.abs(X - ref_x)) <= tol * np.max(np.abs(ref_x))
    assert oracle.solve_backward_error(A, X, B) <= 1e-13

    rfp.rfp_dpftri(transr, uplo, n, arf, info_d[1:2])
    ref_i, info_i = oracle.pftri(transr, uplo, n, ref_f)
    assert info_i == 0 and int(info_d[1].item()) == 0
    got_i = arf.cpu().numpy()
    assert np.max(np.abs(got_i - ref_i)) <= tol * np.max(np.abs(ref_i))
