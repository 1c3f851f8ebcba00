"""rfp_dpfsv_mixed_noalloc (for callers that cannot allocate device memory)
against rfp_dpfsv_mixed with a caller workspace.

Both run the same launch sequence, so the solutions must agree within the
tolerance the mixed-precision tests use (10 * 1e-14 relative to the largest
entry) and both must meet the 1e-14 backward-error bar.  Two calls in a row
share the library's fixed scratch array, which keeps the first call's
contents: the second result must be just as right.  This file is collected
last so that a failure here leaves every other test already run; it passes
alone in a fresh process as well.
"""
import gc

import numpy as np
import pytest

import oracle
import rfp_inputs as gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")


def _inputs(transr, uplo, n, nrhs, seed):
    A, rng = gen.spd_bbt(n, seed=seed, return_rng=True)
    B = gen.rhs(n, nrhs, rng)
    arf = torch.from_numpy(oracle.pack(transr, uplo, A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    return A, B, arf, dB


def _with_workspace(transr, uplo, n, nrhs, arf, dB, prec):
    wb = rfp.rfp_dpfsv_mixed_workspace(n, nrhs, prec)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    X = torch.zeros(nrhs, n, dtype=torch.float64, device="cuda")
    st = torch.zeros(24, dtype=torch.uint8, device="cuda")
    rfp.rfp_dpfsv_mixed(transr, uplo, n, nrhs, arf, dB, n, X, n, prec, 30, 1e-15, work, wb, st)
    return X.cpu().numpy().T, rfp.mixed_status(st.cpu().numpy().tobytes())


def _no_alloc(transr, uplo, n, nrhs, arf, dB, prec):
    X = torch.full((nrhs, n), np.nan, dtype=torch.float64, device="cuda")
    st = torch.zeros(24, dtype=torch.uint8, device="cuda")
    rfp.rfp_dpfsv_mixed_noalloc(transr, uplo, n, nrhs, arf, dB, n, X, n, prec, 30, 1e-15, st)
    return X.cpu().numpy().T, rfp.mixed_status(st.cpu().numpy().tobytes())


def test_no_alloc_matches_workspace_version_twice():
    cases = [("T", "U", 1300, 16, 1, 11),    # TF32 tensor-core panels
             ("N", "L", 900, 5, 2, 12)]      # FP32; reuses the scratch left by the first call
    for transr, uplo, n, nrhs, prec, seed in cases:
        A, B, arf, dB = _inputs(transr, uplo, n, nrhs, seed)
        X_ref, st_ref = _with_workspace(transr, uplo, n, nrhs, arf, dB, prec)
        X, st = _no_alloc(transr, uplo, n, nrhs, arf, dB, prec)
        assert st_ref["converged"] == 1 and st["converged"] == 1, (st_ref, st)
        assert st["info"] == 0 and st["tc_error"] == 0
        assert np.max(np.abs(X - X_ref)) <= 10 * 1e-14 * np.max(np.abs(X_ref))
        assert oracle.solve_backward_error(A, X, B) <= 1e-14


def test_no_alloc_call_allocates_nothing():
    """After a first call (which reserves the fixed array under lazy module
    loading), a further call leaves the device's free memory and the torch
    allocator's count unchanged."""
    transr, uplo, n, nrhs, prec = "N", "U", 700, 3, 2
    A, B, arf, dB = _inputs(transr, uplo, n, nrhs, 21)
    _no_alloc(transr, uplo, n, nrhs, arf, dB, prec)          # set-up call
    X = torch.full((nrhs, n), np.nan, dtype=torch.float64, device="cuda")
    st = torch.zeros(24, dtype=torch.uint8, device="cuda")
    gc.collect()              # temporaries of the set-up call are released now, not mid-test
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    rfp.rfp_dpfsv_mixed_noalloc(transr, uplo, n, nrhs, arf, dB, n, X, n, prec, 30, 1e-15, st)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() <= alloc0
    assert free1 >= free0
    assert rfp.mixed_status(st.cpu().numpy().tobytes())["converged"] == 1
    assert oracle.solve_backward_error(A, X.cpu().numpy().T, B) <= 1e-14


def test_no_alloc_checks_arguments_before_its_capacity():
    st = torch.zeros(24, dtype=torch.uint8, device="cuda")
    big = 4096
    with pytest.raises(rfp.RfpError) as e:      # transr invalid, n too large for the array
        rfp.rfp_dpfsv_mixed_noalloc("X", "L", big, 1, 16, 16, big, 16, big, 2, 5, 1e-14, st)
    assert e.value.status == -1
    with pytest.raises(rfp.RfpError) as e:      # null arf
        rfp.rfp_dpfsv_mixed_noalloc("N", "L", big, 1, 0, 16, big, 16, big, 2, 5, 1e-14, st)
    assert e.value.status == -5


def test_no_alloc_rejects_problems_beyond_its_scratch():
    cap = rfp.rfp_dpfsv_mixed_noalloc_capacity()
    assert cap == 32 << 20
    st = torch.zeros(24, dtype=torch.uint8, device="cuda")
    big = 4096                                   # 4 n^2 bytes alone = 64 MiB
    assert rfp.rfp_dpfsv_mixed_workspace(big, 1, 2) > cap
    with pytest.raises(rfp.RfpError) as e:
        rfp.rfp_dpfsv_mixed_noalloc("N", "L", big, 1, 16, 16, big, 16, big, 2, 5, 1e-14, st)
    assert e.value.status == -3
    n = 2048
    for prec in (0, 1, 2):
        assert rfp.rfp_dpfsv_mixed_workspace(n, 256, prec) <= cap
    assert rfp.rfp_dpfsv_mixed_workspace(1664, 256, 3) <= cap
    assert rfp.rfp_dpfsv_mixed_workspace(1472, 256, 4) <= cap
    assert rfp.rfp_dpfsv_mixed_workspace(n, 1, 3) > cap
    assert rfp.rfp_dpfsv_mixed_workspace(n, 4096, 2) > cap
    with pytest.raises(rfp.RfpError) as e:
        rfp.rfp_dpfsv_mixed_noalloc("N", "L", n, 4096, 16, 16, n, 16, n, 2, 5, 1e-14, st)
    assert e.value.status == -4
