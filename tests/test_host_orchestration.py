"""Host-side orchestration of the CUDA library, checked on the CPU.

The library's host code (``csrc/chol.cu``: the blocked PFTRF / PFTRS /
PFTRI launch sequences, ``csrc/api.cu``: argument checks and the layout
descriptors) is compiled with g++ against ``tests/host_emu``, an emulation of
each kernel launcher with the kernel's own CTA decomposition.  The emulator
fails a launch on any out-of-bounds access and on any element that one CTA
writes while another CTA of the same launch reads or writes it.  So these
tests show, without a GPU, that every launch the library issues stays inside
the caller's buffers, that the in-place steps are race-free, and that the
launch sequences compute what the oracle computes.  The kernels themselves
are tested on the GPU (tests/test_gpu_*.py).
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import rfp_inputs as gen
from paper_0901_1696_gb300.binding import Library, RfpError
from rfp_inputs import LAYOUTS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EMU_DIR = os.path.join(ROOT, "tests", "host_emu")
CSRC = os.path.join(ROOT, "paper_0901_1696_gb300", "csrc")


@pytest.fixture(scope="module")
def emu_lib(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("emu") / "librfp_emu.so")
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-I", EMU_DIR, "-x", "c++",
           os.path.join(CSRC, "chol.cu"), os.path.join(CSRC, "api.cu"),
           os.path.join(CSRC, "mixed.cu"), "-x", "none",
           os.path.join(EMU_DIR, "emu_kernels.cpp"), "-o", so]
    subprocess.run(cmd, check=True)
    lib = Library(so)
    raw = lib.lib
    raw.emu_register.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    raw.emu_message.restype = ctypes.c_char_p
    raw.emu_launches.restype = ctypes.c_long
    raw.emu_set_sms.argtypes = [ctypes.c_int]
    raw.emu_set_step_rules.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_long]
    return lib


@pytest.fixture(params=[152, 1], ids=["sms152", "sms1"])
def emu(emu_lib, request):
    """The emulated device's SM count steers gemm_nt's tile choice: with 152
    SMs many small launches take the small tiles, with 1 SM most launches take
    the large tiles, so both CTA decompositions go through the checks."""
    emu_lib.lib.emu_set_sms(request.param)
    return emu_lib


def _register(emu, *arrays):
    raw = emu.lib
    raw.emu_reset()
    for a in arrays:
        raw.emu_register(a.ctypes.data, a.nbytes)


def _ok(emu):
    raw = emu.lib
    assert raw.emu_violations() == 0, raw.emu_message().decode()


def _full_from_factor(transr, uplo, n, arf):
    F = oracle.unpack(transr, uplo, n, arf)
    return np.tril(F) if uplo == "L" else np.triu(F).T


SIZES = [1, 2, 3, 5, 63, 64, 65, 127, 128, 129, 200, 257, 400]


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", SIZES)
def test_emulated_path_matches_oracle(emu, transr, uplo, n):
    A, rng = gen.spd_bbt(n, seed=n + 7, return_rng=True)
    nrhs = 3 if n % 2 else 70
    B = gen.rhs(n, nrhs, rng)
    lda = n + 3
    Afull = np.zeros((lda, n), order="F")
    Afull[:n] = A
    arf = np.zeros(n * (n + 1) // 2)
    info = np.zeros(1, dtype=np.int32)
    ldb = n + 1
    Bw = np.zeros((ldb, nrhs), order="F")
    Bw[:n] = B
    _register(emu, Afull, arf, info, Bw)

    emu.rfp_dpack(transr, uplo, n, Afull, lda, arf, 0)
    _ok(emu)
    np.testing.assert_array_equal(arf, oracle.pack(transr, uplo, A))

    ref_f, ref_info = oracle.pftrf(transr, uplo, n, arf)
    emu.rfp_dpftrf(transr, uplo, n, arf, info, 0)
    _ok(emu)
    assert info[0] == ref_info == 0
    assert np.max(np.abs(arf - ref_f)) <= 1e-13 * max(1.0, np.max(np.abs(ref_f)))

    X = oracle.pftrs(transr, uplo, n, arf, B)
    emu.rfp_dpftrs(transr, uplo, n, nrhs, arf, Bw, ldb, 0)
    _ok(emu)
    assert np.max(np.abs(Bw[:n] - X)) <= 1e-12 * max(1.0, np.max(np.abs(X)))

    ref_i, _ = oracle.pftri(transr, uplo, n, arf)
    emu.rfp_dpftri(transr, uplo, n, arf, info, 0)
    _ok(emu)
    assert info[0] == 0
    assert np.max(np.abs(arf - ref_i)) <= 1e-12 * max(1.0, np.max(np.abs(ref_i)))

    # unpack writes the UPLO triangle only
    Aout = np.full((lda, n), 7.0, order="F")
    _register(emu, Aout, arf)
    emu.rfp_dunpack(transr, uplo, n, arf, Aout, lda, 0)
    _ok(emu)
    want = oracle.unpack(transr, uplo, n, arf, np.full((n, n), 7.0))
    np.testing.assert_array_equal(Aout[:n], want)
    assert np.all(Aout[n:] == 7.0)


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [129, 258, 400])
@pytest.mark.parametrize("rules", [(0, 0, 0), (0, 4096, 0), (4096, 0, 0), (4096, 2048, 64),
                                   (0, 0, 64), (0, 4096, 32)],
                         ids=["panel64_strip64", "panel64_strip32", "panel32_strip64",
                              "panel32_bulk64", "panel64_bulk64", "panel64_strip32_bulk32"])
def test_emulated_step_rules(emu_lib, transr, uplo, n, rules):
    """The lookahead steps with 64-wide panels (the rule for triangles above
    order 4096), 32-wide panels with 64-row strips (orders 2049 .. 4096), and
    either bulk tile width, at orders the emulator covers: same bounds,
    ownership and ordering checks, same factor as the oracle."""
    raw = emu_lib.lib
    raw.emu_set_sms(152)
    raw.emu_set_step_rules(*rules)
    try:
        A = gen.spd_bbt(n, seed=n + 11)
        arf = oracle.pack(transr, uplo, A)
        info = np.zeros(1, dtype=np.int32)
        _register(emu_lib, arf, info)
        ref_f, ref_info = oracle.pftrf(transr, uplo, n, arf)
        emu_lib.rfp_dpftrf(transr, uplo, n, arf, info, 0)
        _ok(emu_lib)
        assert info[0] == ref_info == 0
        assert np.max(np.abs(arf - ref_f)) <= 1e-13 * max(1.0, np.max(np.abs(ref_f)))
    finally:
        raw.emu_set_step_rules(4096, 2048, 0)


@pytest.mark.parametrize("transr,uplo", [("N", "L"), ("T", "U")])
def test_emulated_split_k_updates(emu_lib, transr, uplo):
    """n = 530: PFTRF step 3 and PFTRI's T1 update have K = 265 and few
    output tiles, so they run as split-K products (chunks into scratch, summed
    by a second kernel), checked like every other launch."""
    n = 530
    raw = emu_lib.lib
    raw.emu_set_sms(152)
    A = gen.spd_bbt(n, seed=17)
    arf = oracle.pack(transr, uplo, A)
    info = np.zeros(1, dtype=np.int32)
    _register(emu_lib, arf, info)
    ref_f, _ = oracle.pftrf(transr, uplo, n, arf)
    emu_lib.rfp_dpftrf(transr, uplo, n, arf, info, 0)
    _ok(emu_lib)
    assert info[0] == 0
    assert np.max(np.abs(arf - ref_f)) <= 1e-13 * max(1.0, np.max(np.abs(ref_f)))
    ref_i, _ = oracle.pftri(transr, uplo, n, arf)
    emu_lib.rfp_dpftri(transr, uplo, n, arf, info, 0)
    _ok(emu_lib)
    assert info[0] == 0
    assert np.max(np.abs(arf - ref_i)) <= 1e-12 * max(1.0, np.max(np.abs(ref_i)))


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [7, 130])
def test_emulated_single_precision(emu, transr, uplo, n):
    A, rng = gen.spd_bbt(n, seed=3, return_rng=True)
    B = gen.rhs(n, 5, rng)
    A32 = np.asfortranarray(A.astype(np.float32))
    arf = np.zeros(n * (n + 1) // 2, dtype=np.float32)
    info = np.zeros(1, dtype=np.int32)
    B32 = np.asfortranarray(B.astype(np.float32))
    _register(emu, A32, arf, info, B32)
    emu.rfp_spack(transr, uplo, n, A32, n, arf, 0)
    np.testing.assert_array_equal(arf, oracle.pack(transr, uplo, A32.astype(np.float64)))
    emu.rfp_spftrf(transr, uplo, n, arf, info, 0)
    emu.rfp_spftrs(transr, uplo, n, 5, arf, B32, n, 0)
    _ok(emu)
    assert info[0] == 0
    assert oracle.solve_backward_error(A, B32.astype(np.float64), B) <= 64 * n * 6e-8


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n,k", [(70, 3), (70, 40), (130, 64), (130, 100), (300, 100), (300, 140),
                                 (300, 260), (300, 200)])
def test_emulated_info_on_failure(emu, transr, uplo, n, k):
    A, L0 = gen.spd_integer_factor(n, seed=5)
    A = A.copy()
    A[k, k] -= L0[k, k] ** 2 + 1.0
    arf = oracle.pack(transr, uplo, A)
    info = np.zeros(1, dtype=np.int32)
    _register(emu, arf, info)
    emu.rfp_dpftrf(transr, uplo, n, arf, info, 0)
    _ok(emu)
    assert info[0] == k + 1


def test_emulated_pftri_zero_diagonal(emu):
    n = 90
    arf = oracle.pack("N", "L", np.diag(np.r_[np.ones(70), 0.0, np.ones(19)]))
    info = np.zeros(1, dtype=np.int32)
    _register(emu, arf, info)
    emu.rfp_dpftri("N", "L", n, arf, info, 0)
    _ok(emu)
    assert info[0] == 71


@pytest.mark.parametrize("n", [0, 1, 2, 6, 7, 100, 1001])
@pytest.mark.parametrize("transr,uplo", LAYOUTS)
def test_layout_descriptor_matches_oracle_placement(emu, transr, uplo, n):
    """rfp_layout's block descriptors place every element where the oracle's
    block assembly (Figs. 4-6) puts it: bit-exact index work."""
    d = emu.rfp_layout(transr, uplo, n)
    n1, n2, ld = d["n1"], d["n2"], d["ld"]
    assert (n1, n2) == oracle.split(uplo, n)
    code = np.zeros((n, n), order="F")
    for j in range(n):
        for i in range(n):
            code[i, j] = 1 + i + j * n
    arf = oracle.pack(transr, uplo, code)
    for (off, tr, rows, cols, r0, c0, tri) in [
            (d["t1_off"], d["t1_trans"], n1, n1, 0, 0, True),
            (d["s_off"], d["s_trans"], n2, n1, n1, 0, False),
            (d["t2_off"], d["t2_trans"], n2, n2, n1, n1, True)]:
        for i in range(rows):
            for j in range(i + 1 if tri else cols):
                pos = off + (j + i * ld if tr else i + j * ld)
                gi, gj = r0 + i, c0 + j          # logical lower element
                a = code[gi, gj] if uplo == "L" else code[gj, gi]
                assert arf[pos] == a


def test_argument_checks(emu):
    arf = np.zeros(10)
    info = np.zeros(1, dtype=np.int32)
    B = np.zeros((4, 2), order="F")
    cases = [
        (lambda: emu.rfp_dpftrf("X", "L", 4, arf, info, 0), -1),
        (lambda: emu.rfp_dpftrf("N", "C", 4, arf, info, 0), -2),
        (lambda: emu.rfp_dpftrf("N", "L", -1, arf, info, 0), -3),
        (lambda: emu.rfp_dpftrf("N", "L", 4, 0, info, 0), -4),
        (lambda: emu.rfp_dpftrf("N", "L", 4, arf, 0, 0), -5),
        (lambda: emu.rfp_dpftrf("N", "L", 4, arf.ctypes.data + 1, info, 0), -4),
        (lambda: emu.rfp_dpftrs("N", "L", 4, -2, arf, B, 4, 0), -4),
        (lambda: emu.rfp_dpftrs("N", "L", 4, 2, 0, B, 4, 0), -5),
        (lambda: emu.rfp_dpftrs("N", "L", 4, 2, arf, B, 3, 0), -7),
        (lambda: emu.rfp_dpack("T", "U", 4, B, 3, arf, 0), -5),
        (lambda: emu.rfp_dunpack("T", "U", 4, arf, B, 2, 0), -6),
        (lambda: emu.rfp_dpftri("c", "L", 4, arf, info, 0), -1),
    ]
    for call, code in cases:
        with pytest.raises(RfpError) as e:
            call()
        assert e.value.status == code
    # quick returns
    assert emu.rfp_dpftrs("N", "L", 0, 5, 0, 0, 1, 0) == 0
    assert emu.rfp_dpftrs("N", "L", 4, 0, 0, 0, 4, 0) == 0
    assert emu.rfp_dpack("N", "L", 0, 0, 1, 0, 0) == 0


def _aligned_bytes(nbytes, align=256):
    raw = np.zeros(nbytes + align, dtype=np.uint8)
    off = (-raw.ctypes.data) % align
    return raw[off:off + nbytes]


@pytest.mark.parametrize("prec", [2, 3, 4, 1, 0], ids=["fp32", "tf32x3", "bf16x6", "tf32", "bf16"])
@pytest.mark.parametrize("transr,uplo,n", [("N", "L", 5), ("T", "U", 70), ("N", "U", 600),
                                           ("T", "L", 600)])
def test_emulated_mixed_precision_solve(emu_lib, prec, transr, uplo, n):
    """The refinement loop's launch sequence, in bounds and race-free, reaches
    an FP64-accurate solution (n = 600 runs one 512-wide panel and one
    tensor-core SYRK update)."""
    from paper_0901_1696_gb300.binding import mixed_status
    emu = emu_lib
    emu.lib.emu_set_sms(152)
    if n == 600 and prec == 2 and transr == "T":
        pytest.skip("the FP32 path has no panel split; one 600 case is enough")
    A, rng = gen.spd_bbt(n, seed=n, return_rng=True)
    nrhs = 3
    B = gen.rhs(n, nrhs, rng)
    arf = oracle.pack(transr, uplo, A)
    X = np.zeros((n + 2, nrhs), order="F")
    wbytes = emu.rfp_dpfsv_mixed_workspace(n, nrhs, prec)
    work = _aligned_bytes(wbytes)
    status = _aligned_bytes(24, 8)
    Bc = np.asfortranarray(B)
    _register(emu, arf, Bc, X, work, status)
    emu.rfp_dpfsv_mixed(transr, uplo, n, nrhs, arf, Bc, n, X, n + 2, prec, 10, 1e-15, work,
                        wbytes, status, 0)
    _ok(emu)
    st = mixed_status(status.tobytes())
    assert st["info"] == 0 and st["tc_error"] == 0
    assert st["converged"] == 1 and 1 <= st["iterations"] <= 6, st
    assert oracle.solve_backward_error(A, X[:n], B) <= 1e-15
    np.testing.assert_array_equal(arf, oracle.pack(transr, uplo, A))   # A untouched


@pytest.mark.parametrize("transr,uplo,n", [("N", "L", 600), ("T", "U", 257)])
def test_emulated_one_step_is_one_fp32_solve(emu_lib, transr, uplo, n):
    """max_iter = 1 returns X = (L L^T)^{-1} fl32(B) from the FP32 factor: the
    block solves alone (several 128-row blocks, a ragged last block, two
    column groups of which the second is ragged) against the oracle's solve."""
    from paper_0901_1696_gb300.binding import mixed_status
    emu = emu_lib
    emu.lib.emu_set_sms(152)
    A, rng = gen.spd_bbt(n, seed=n + 1, return_rng=True)
    nrhs = 20
    B = gen.rhs(n, nrhs, rng)
    arf = oracle.pack(transr, uplo, A)
    X = np.zeros((n, nrhs), order="F")
    wbytes = emu.rfp_dpfsv_mixed_workspace(n, nrhs, 2)
    work = _aligned_bytes(wbytes)
    status = _aligned_bytes(24, 8)
    Bc = np.asfortranarray(B)
    _register(emu, arf, Bc, X, work, status)
    emu.rfp_dpfsv_mixed(transr, uplo, n, nrhs, arf, Bc, n, X, n, 2, 1, 1e-15, work, wbytes,
                        status, 0)
    _ok(emu)
    st = mixed_status(status.tobytes())
    assert st["info"] == 0 and st["tc_error"] == 0 and st["iterations"] == 1, st
    ref = oracle.pftrs(transr, uplo, n, oracle.pftrf(transr, uplo, n, arf)[0], B)
    assert np.max(np.abs(X - ref)) <= 1e-4 * np.max(np.abs(ref))


# ---- the rest of the LAPACK 3.2 RFP routine set, emulated ----

def _triangle_arf(transr, uplo, n, seed):
    """A well-conditioned triangle in RFP: the Cholesky factor of B B^T / n + I."""
    L = np.linalg.cholesky(gen.spd_bbt(n, seed=seed))
    return oracle.pack(transr, uplo, L if uplo == "L" else L.T)


@pytest.mark.parametrize("transr,uplo", LAYOUTS)
@pytest.mark.parametrize("n", [1, 5, 64, 130, 201])
def test_emulated_surface_routines(emu_lib, transr, uplo, n):
    emu = emu_lib
    emu.lib.emu_set_sms(152)
    rng = np.random.default_rng(n)
    nt = n * (n + 1) // 2
    # TPTTF / TFTTP: bit-exact
    ap = rng.standard_normal(nt)
    arf = np.zeros(nt)
    back = np.zeros(nt)
    _register(emu, ap, arf, back)
    emu.rfp_dtpttf(transr, uplo, n, ap, arf, 0)
    emu.rfp_dtfttp(transr, uplo, n, arf, back, 0)
    _ok(emu)
    np.testing.assert_array_equal(arf, oracle.tpttf(transr, uplo, n, ap))
    np.testing.assert_array_equal(back, ap)
    # TFTRI, both diagonal kinds
    for diag in "NU":
        tri = _triangle_arf(transr, uplo, n, seed=n + 1)
        ref, ref_info = oracle.tftri(transr, uplo, diag, n, tri)
        work = np.zeros(n)
        info = np.zeros(1, dtype=np.int32)
        _register(emu, tri, work, info)
        emu.rfp_dtftri(transr, uplo, diag, n, tri, info, work, 0)
        _ok(emu)
        assert info[0] == ref_info == 0
        assert np.max(np.abs(tri - ref)) <= 1e-12 * np.max(np.abs(ref))
    # SFRK
    for trans, k in (("N", 7), ("T", 70)):
        A = rng.standard_normal((n, k) if trans == "N" else (k, n))
        Af = np.asfortranarray(A)
        C = rng.standard_normal((n, n))
        C = oracle.pack(transr, uplo, C + C.T)
        ref = oracle.sfrk(transr, uplo, trans, n, k, 0.5, A, -2.0, C)
        _register(emu, Af, C)
        emu.rfp_dsfrk(transr, uplo, trans, n, k, 0.5, Af, A.shape[0], -2.0, C, 0)
        _ok(emu)
        assert np.max(np.abs(C - ref)) <= 1e-13 * np.max(np.abs(ref))
    # TFSM, every side / trans / diag
    tri = _triangle_arf(transr, uplo, n, seed=n + 2)
    for side in "LR":
        for trans in "NT":
            for diag in "NU":
                m, nc = (n, 3) if side == "L" else (4, n)
                B = rng.standard_normal((m, nc))
                ldb = m + 2
                Bw = np.zeros((ldb, nc), order="F")
                Bw[:m] = B
                ref = oracle.tfsm(transr, side, uplo, trans, diag, m, nc, 1.25, tri, B)
                _register(emu, tri, Bw)
                emu.rfp_dtfsm(transr, side, uplo, trans, diag, m, nc, 1.25, tri, Bw, ldb, 0)
                _ok(emu)
                assert np.max(np.abs(Bw[:m] - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref))), \
                    (side, trans, diag)
    # LANSF
    S = rng.standard_normal((n, n))
    sarf = oracle.pack(transr, uplo, S + S.T)
    work = np.zeros(2 * n)
    val = np.zeros(1)
    for norm in "M1OIFE":
        _register(emu, sarf, work, val)
        emu.rfp_dlansf(norm, transr, uplo, n, sarf, work, val, 0)
        _ok(emu)
        ref = oracle.lansf(norm, transr, uplo, n, sarf)
        assert abs(val[0] - ref) <= 1e-14 * ref, norm


def test_emulated_surface_edge_cases(emu_lib):
    """Empty sizes return at once without touching memory; alpha = 0 and
    k = 0 follow LAPACK (B := 0, C := beta C); leading dimensions above the
    order leave the padding untouched."""
    emu = emu_lib
    emu.lib.emu_set_sms(152)
    z = np.zeros(4)
    info = np.zeros(1, dtype=np.int32)
    _register(emu, z, info)
    for f in (lambda: emu.rfp_dtpttf("N", "L", 0, z, z, 0),
              lambda: emu.rfp_dtfttp("T", "U", 0, z, z, 0),
              lambda: emu.rfp_dtfsm("N", "L", "L", "N", "N", 0, 3, 1.0, z, z, 1, 0),
              lambda: emu.rfp_dtfsm("N", "R", "U", "T", "U", 3, 0, 1.0, z, z, 3, 0),
              lambda: emu.rfp_dsfrk("N", "L", "N", 0, 5, 1.0, z, 1, 0.0, z, 0)):
        assert f() == 0
    emu.rfp_dtftri("N", "L", "N", 0, z, info, None, 0)
    _ok(emu)
    assert info[0] == 0
    # SFRK with k = 0: C := beta C, A not read (null)
    n = 9
    rng = np.random.default_rng(1)
    S = rng.standard_normal((n, n))
    for t, u in LAYOUTS:
        C = oracle.pack(t, u, S + S.T)
        ref = oracle.sfrk(t, u, "N", n, 0, 1.0, np.zeros((n, 0)), -0.5, C)
        _register(emu, C)
        emu.rfp_dsfrk(t, u, "N", n, 0, 1.0, None, n, -0.5, C, 0)
        _ok(emu)
        np.testing.assert_allclose(C, ref, rtol=0, atol=1e-15)
    # TFSM with alpha = 0: B := 0 and A is not read (null); ldb padding untouched
    m, nc, ldb = 7, 3, 10
    Bw = np.full((ldb, nc), 5.0, order="F")
    _register(emu, Bw)
    emu.rfp_dtfsm("T", "L", "U", "N", "N", m, nc, 0.0, None, Bw, ldb, 0)
    _ok(emu)
    assert np.array_equal(Bw[:m], np.zeros((m, nc))) and np.array_equal(Bw[m:], np.full((ldb - m, nc), 5.0))
    # SFRK with lda above the order
    k, lda = 4, n + 3
    A = np.zeros((lda, k), order="F")
    A[:n] = rng.standard_normal((n, k))
    C = oracle.pack("N", "U", np.eye(n))
    ref = oracle.sfrk("N", "U", "N", n, k, 2.0, A[:n], 1.0, C)
    _register(emu, A, C)
    emu.rfp_dsfrk("N", "U", "N", n, k, 2.0, A, lda, 1.0, C, 0)
    _ok(emu)
    np.testing.assert_allclose(C, ref, rtol=0, atol=1e-13)
