"""Guard canaries on the GPU: every RFP array, right-hand side, solution and
workspace is placed between NaN guard words, and after the calls the guards
must still be NaN (no kernel writes outside its buffers)."""
import numpy as np
import pytest

import oracle
import rfp_inputs as gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rfp = pytest.importorskip("paper_0901_1696_gb300.binding")

G = 64   # guard elements on each side (512 bytes in FP64: alignment is kept)
LAYOUTS = [(t, u) for t in "NT" for u in "LU"]


def guarded(values, dtype=torch.float64):
    """(full buffer, inner view) with NaN guards around `values`."""
    v = torch.as_tensor(np.ascontiguousarray(values)).to("cuda", dtype).reshape(-1)
    buf = torch.full((v.numel() + 2 * G,), float("nan"), dtype=dtype, device="cuda")
    buf[G:G + v.numel()] = v
    return buf, buf[G:G + v.numel()]


def guards_intact(buf):
    return bool(torch.isnan(buf[:G]).all() and torch.isnan(buf[-G:]).all())


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [1, 64, 65, 513])
def test_fp64_routines_stay_inside_their_buffers(transr, uplo, n):
    A, rng = gen.spd_bbt(n, seed=n, return_rng=True)
    nrhs, ldb = 3, n + 2
    Abuf, Ad = guarded(np.asfortranarray(A).ravel(order="F"))
    arfbuf, arf = guarded(np.zeros(n * (n + 1) // 2))
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    Bw = np.zeros((ldb, nrhs))
    Bw[:n] = gen.rhs(n, nrhs, rng)
    Bbuf, Bd = guarded(Bw.T)                                  # column-major, ld = ldb
    rfp.rfp_dpack(transr, uplo, n, Ad, n, arf)
    rfp.rfp_dpftrf(transr, uplo, n, arf, info)
    rfp.rfp_dpftrs(transr, uplo, n, nrhs, arf, Bd, ldb)
    rfp.rfp_dpftri(transr, uplo, n, arf, info)
    rfp.rfp_dunpack(transr, uplo, n, arf, Ad, n)
    apbuf, ap = guarded(np.zeros(n * (n + 1) // 2))
    rfp.rfp_dtfttp(transr, uplo, n, arf, ap)
    rfp.rfp_dtpttf(transr, uplo, n, ap, arf)
    wbuf, work = guarded(np.zeros(2 * n))
    vbuf, val = guarded(np.zeros(1))
    rfp.rfp_dlansf("F", transr, uplo, n, arf, work, val)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    for b in (Abuf, arfbuf, Bbuf, apbuf, wbuf, vbuf):
        assert guards_intact(b)


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
def test_mixed_and_batched_stay_inside_their_buffers(transr, uplo):
    n, nrhs = 700, 4
    A, rng = gen.spd_bbt(n, seed=3, return_rng=True)
    B = gen.rhs(n, nrhs, rng)
    arfbuf, arf = guarded(oracle.pack(transr, uplo, A))
    Bbuf, Bd = guarded(B.T)
    Xbuf, Xd = guarded(np.zeros((nrhs, n)))
    for prec in (rfp.RFP_PREC_FP32, rfp.RFP_PREC_TF32X3, rfp.RFP_PREC_BF16X6):
        wb = rfp.rfp_dpfsv_mixed_workspace(n, nrhs, prec)
        # the workspace must be 256-byte aligned: guards of 256 bytes each side
        wbuf = torch.full((wb + 512,), 0x7F, dtype=torch.uint8, device="cuda")
        status = torch.zeros(24, dtype=torch.uint8, device="cuda")
        rfp.rfp_dpfsv_mixed(transr, uplo, n, nrhs, arf, Bd, n, Xd, n, prec, 30, 1e-15,
                            wbuf[256:256 + wb], wb, status)
        torch.cuda.synchronize()
        assert bool((wbuf[:256] == 0x7F).all() and (wbuf[256 + wb:] == 0x7F).all()), prec
        for b in (arfbuf, Bbuf, Xbuf):
            assert guards_intact(b)
    # batched: three matrices back to back inside one guarded buffer
    ns, nr = [5, 300, 512], [2, 8, 1]
    from paper_0901_1696_gb300 import batched as bt
    e, al, bl = bt.make_entries(ns, [transr] * 3, [uplo] * 3, nr)
    arfs = np.concatenate([oracle.pack(transr, uplo, gen.spd_bbt(m, seed=m)) for m in ns])
    aall_buf, aall = guarded(arfs)
    ball_buf, ball = guarded(np.ones(bl))
    plan = torch.empty(rfp.rfp_batch_plan_bytes(3), dtype=torch.uint8, device="cuda")
    rfp.rfp_batch_plan(3, e, al, bl, plan, plan.numel())
    infos = torch.zeros(3, dtype=torch.int32, device="cuda")
    rfp.rfp_dpfsv_batched(3, plan, aall, ball, infos)
    torch.cuda.synchronize()
    assert int(infos.abs().sum().item()) == 0
    assert guards_intact(aall_buf) and guards_intact(ball_buf)
