"""Thin ctypes binding of the C ABI in include/rfp.h (argument marshalling only).

Every function has the name of its C entry point and takes the same
arguments in the same order.  Array arguments may be torch CUDA tensors
(their data_ptr is passed), numpy arrays (their buffer address; used only by
host-side tests) or plain integers (addresses).  ``stream=None`` means the
current torch CUDA stream.  A non-zero return code raises RfpError carrying
the code; nothing is computed here.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_LIB = os.path.join(_HERE, "_build", "librfp_gb300.so")


class RfpError(RuntimeError):
    def __init__(self, func: str, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"{func} returned {status}: {detail}")


class RfpLayout(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n1", ctypes.c_int64), ("n2", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("t1_off", ctypes.c_int64), ("s_off", ctypes.c_int64),
                ("t2_off", ctypes.c_int64), ("t1_trans", ctypes.c_int32),
                ("s_trans", ctypes.c_int32), ("t2_trans", ctypes.c_int32)]


_c, _i64, _p, _i32p = ctypes.c_char, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
SIGNATURES = {
    "rfp_layout": [_c, _c, _i64, ctypes.POINTER(RfpLayout)],
    "rfp_dpack": [_c, _c, _i64, _p, _i64, _p, _p],
    "rfp_spack": [_c, _c, _i64, _p, _i64, _p, _p],
    "rfp_dunpack": [_c, _c, _i64, _p, _p, _i64, _p],
    "rfp_sunpack": [_c, _c, _i64, _p, _p, _i64, _p],
    "rfp_dpftrf": [_c, _c, _i64, _p, _i32p, _p],
    "rfp_spftrf": [_c, _c, _i64, _p, _i32p, _p],
    "rfp_dpftrs": [_c, _c, _i64, _i64, _p, _p, _i64, _p],
    "rfp_spftrs": [_c, _c, _i64, _i64, _p, _p, _i64, _p],
    "rfp_dpftri": [_c, _c, _i64, _p, _i32p, _p],
    "rfp_spftri": [_c, _c, _i64, _p, _i32p, _p],
    "rfp_dpfsv_mixed": [_c, _c, _i64, _i64, _p, _p, _i64, _p, _i64, ctypes.c_int, ctypes.c_int,
                        ctypes.c_double, _p, ctypes.c_size_t, _p, _p],
    "rfp_ssyrk_tc": [_c, _i64, _i64, ctypes.c_float, _p, _i64, ctypes.c_int, ctypes.c_float, _p,
                     _i64, _i32p, _p],
}
for _x, _f in (("d", ctypes.c_double), ("s", ctypes.c_float)):
    SIGNATURES.update({
        f"rfp_{_x}tpttf": [_c, _c, _i64, _p, _p, _p],
        f"rfp_{_x}tfttp": [_c, _c, _i64, _p, _p, _p],
        f"rfp_{_x}tftri": [_c, _c, _c, _i64, _p, _i32p, _p, _p],
        f"rfp_{_x}sfrk": [_c, _c, _c, _i64, _i64, _f, _p, _i64, _f, _p, _p],
        f"rfp_{_x}tfsm": [_c, _c, _c, _c, _c, _i64, _i64, _f, _p, _p, _i64, _p],
        f"rfp_{_x}lansf": [_c, _c, _c, _i64, _p, _p, _p, _p],
    })
RFP_PREC_BF16, RFP_PREC_TF32, RFP_PREC_FP32, RFP_PREC_TF32X3, RFP_PREC_BF16X6 = 0, 1, 2, 3, 4


class RfpMixedStatus(ctypes.Structure):
    _fields_ = [("info", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("tc_error", ctypes.c_int32),
                ("backward_error", ctypes.c_double)]


def batch_entry_dtype():
    """numpy dtype with the layout of rfp_batch_entry_t (40 bytes)."""
    import numpy as np
    return np.dtype([("n", "<i8"), ("arf", "<i8"), ("b", "<i8"), ("nrhs", "<i4"), ("ldb", "<i4"),
                     ("transr", "S1"), ("uplo", "S1"), ("nb", "<i2"), ("reserved", "<i4")])


def mixed_status(raw: bytes) -> dict:
    """Decode the 24-byte rfp_mixed_status_t read back from the device."""
    st = RfpMixedStatus.from_buffer_copy(bytes(raw))
    return {f: getattr(st, f) for f, _ in RfpMixedStatus._fields_}


def _addr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):          # torch tensor
        return x.data_ptr()
    if hasattr(x, "ctypes"):            # numpy array
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream                # torch.cuda.Stream


def _ch(c: str) -> bytes:
    return c.encode()[:1] if isinstance(c, str) else bytes(c[:1])


class Library:
    """One loaded copy of the C ABI (the CUDA build by default)."""

    def __init__(self, path: str = DEFAULT_LIB):
        if not os.path.exists(path):
            raise RuntimeError(
                f"RFP CUDA library not found at {path}; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        self.path = path
        self.lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            f = getattr(self.lib, name)
            f.argtypes, f.restype = args, ctypes.c_int
        self.lib.rfp_status_string.argtypes, self.lib.rfp_status_string.restype = [ctypes.c_int], ctypes.c_char_p
        self.lib.rfp_last_cuda_error.argtypes, self.lib.rfp_last_cuda_error.restype = [], ctypes.c_char_p
        self.lib.rfp_kernel_launches.argtypes, self.lib.rfp_kernel_launches.restype = [], ctypes.c_int64
        self.lib.rfp_stage_timing.argtypes, self.lib.rfp_stage_timing.restype = [ctypes.c_int], ctypes.c_int
        self.lib.rfp_stage_times.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(ctypes.c_char_p)]
        self.lib.rfp_stage_times.restype = ctypes.c_int

    def _check(self, name: str, rc: int) -> int:
        if rc != 0:
            detail = self.lib.rfp_status_string(rc).decode()
            if rc > 0:
                detail += f" ({self.lib.rfp_last_cuda_error().decode()})"
            raise RfpError(name, rc, detail)
        return rc

    def rfp_kernel_launches(self) -> int:
        return int(self.lib.rfp_kernel_launches())

    def rfp_stage_timing(self, enable: bool):
        return self._check("rfp_stage_timing", self.lib.rfp_stage_timing(1 if enable else 0))

    def rfp_stage_times(self, max_stages: int = 8192):
        """[(step name, ms), ...] of every call timed since rfp_stage_timing."""
        ms = (ctypes.c_float * max_stages)()
        names = (ctypes.c_char_p * max_stages)()
        k = self.lib.rfp_stage_times(max_stages, ms, names)
        if k < 0:
            raise RfpError("rfp_stage_times", -k, self.lib.rfp_last_cuda_error().decode())
        return [(names[i].decode(), float(ms[i])) for i in range(k)]

    def rfp_layout(self, transr, uplo, n):
        out = RfpLayout()
        self._check("rfp_layout", self.lib.rfp_layout(_ch(transr), _ch(uplo), n, ctypes.byref(out)))
        return {f: getattr(out, f) for f, _ in RfpLayout._fields_}

    def _pack(self, name, transr, uplo, n, x, ld_or_y, y_or_ld, stream):
        f = getattr(self.lib, name)
        if "unpack" in name:     # (arf, A, lda)
            rc = f(_ch(transr), _ch(uplo), n, _addr(x), _addr(ld_or_y), y_or_ld, _stream(stream))
        else:                    # (A, lda, arf)
            rc = f(_ch(transr), _ch(uplo), n, _addr(x), ld_or_y, _addr(y_or_ld), _stream(stream))
        return self._check(name, rc)

    def rfp_dpack(self, transr, uplo, n, A, lda, arf, stream=None):
        return self._pack("rfp_dpack", transr, uplo, n, A, lda, arf, stream)

    def rfp_spack(self, transr, uplo, n, A, lda, arf, stream=None):
        return self._pack("rfp_spack", transr, uplo, n, A, lda, arf, stream)

    def rfp_dunpack(self, transr, uplo, n, arf, A, lda, stream=None):
        return self._pack("rfp_dunpack", transr, uplo, n, arf, A, lda, stream)

    def rfp_sunpack(self, transr, uplo, n, arf, A, lda, stream=None):
        return self._pack("rfp_sunpack", transr, uplo, n, arf, A, lda, stream)

    def _fac(self, name, transr, uplo, n, arf, info, stream):
        rc = getattr(self.lib, name)(_ch(transr), _ch(uplo), n, _addr(arf), _addr(info),
                                     _stream(stream))
        return self._check(name, rc)

    def rfp_dpftrf(self, transr, uplo, n, arf, info, stream=None):
        return self._fac("rfp_dpftrf", transr, uplo, n, arf, info, stream)

    def rfp_spftrf(self, transr, uplo, n, arf, info, stream=None):
        return self._fac("rfp_spftrf", transr, uplo, n, arf, info, stream)

    def rfp_dpftri(self, transr, uplo, n, arf, info, stream=None):
        return self._fac("rfp_dpftri", transr, uplo, n, arf, info, stream)

    def rfp_spftri(self, transr, uplo, n, arf, info, stream=None):
        return self._fac("rfp_spftri", transr, uplo, n, arf, info, stream)

    def _trs(self, name, transr, uplo, n, nrhs, arf, B, ldb, stream):
        rc = getattr(self.lib, name)(_ch(transr), _ch(uplo), n, nrhs, _addr(arf), _addr(B), ldb,
                                     _stream(stream))
        return self._check(name, rc)

    def rfp_dpfsv_mixed_workspace(self, n, nrhs, prec) -> int:
        f = self.lib.rfp_dpfsv_mixed_workspace
        f.argtypes, f.restype = [_i64, _i64, ctypes.c_int], ctypes.c_size_t
        return int(f(n, nrhs, prec))

    def rfp_dpfsv_mixed(self, transr, uplo, n, nrhs, arf, B, ldb, X, ldx, prec, max_iter, tol,
                        work, work_bytes, status, stream=None):
        rc = self.lib.rfp_dpfsv_mixed(_ch(transr), _ch(uplo), n, nrhs, _addr(arf), _addr(B), ldb,
                                      _addr(X), ldx, prec, max_iter, tol, _addr(work), work_bytes,
                                      _addr(status), _stream(stream))
        return self._check("rfp_dpfsv_mixed", rc)

    def rfp_dpfsv_mixed_noalloc_capacity(self) -> int:
        f = self.lib.rfp_dpfsv_mixed_noalloc_capacity
        f.argtypes, f.restype = [], ctypes.c_size_t
        return int(f())

    def rfp_dpfsv_mixed_noalloc(self, transr, uplo, n, nrhs, arf, B, ldb, X, ldx, prec, max_iter,
                                tol, status, stream=None):
        f = self.lib.rfp_dpfsv_mixed_noalloc
        f.argtypes = [_c, _c, _i64, _i64, _p, _p, _i64, _p, _i64, ctypes.c_int, ctypes.c_int,
                      ctypes.c_double, _p, _p]
        f.restype = ctypes.c_int
        rc = f(_ch(transr), _ch(uplo), n, nrhs, _addr(arf), _addr(B), ldb, _addr(X), ldx, prec,
               max_iter, tol, _addr(status), _stream(stream))
        return self._check("rfp_dpfsv_mixed_noalloc", rc)

    def rfp_batch_plan_bytes(self, batch) -> int:
        f = self.lib.rfp_batch_plan_bytes
        f.argtypes, f.restype = [_i64], ctypes.c_size_t
        return int(f(batch))

    def rfp_batch_plan(self, batch, entries, arf_len, b_len, d_plan, plan_bytes, stream=None):
        """entries: numpy array of batch_entry_dtype(); returns the bad entry
        index (-1 if none) when the plan is rejected with -2 (raises)."""
        f = self.lib.rfp_batch_plan
        f.argtypes = [_i64, _p, _i64, _i64, _p, ctypes.c_size_t, _p, _p]
        f.restype = ctypes.c_int
        bad = ctypes.c_int64(-1)
        rc = f(batch, _addr(entries), arf_len, b_len, _addr(d_plan), plan_bytes,
               ctypes.addressof(bad), _stream(stream))
        if rc == -2:
            raise RfpError("rfp_batch_plan", rc, f"entry {bad.value} is invalid")
        return self._check("rfp_batch_plan", rc)

    def _batched(self, name, batch, d_plan, arf, B, d_info, stream):
        f = getattr(self.lib, name)
        f.argtypes = [_i64, _p, _p, _p, _p, _p]
        f.restype = ctypes.c_int
        return self._check(name, f(batch, _addr(d_plan), _addr(arf), _addr(B), _addr(d_info),
                                   _stream(stream)))

    def rfp_dpfsv_batched(self, batch, d_plan, arf, B, d_info, stream=None):
        return self._batched("rfp_dpfsv_batched", batch, d_plan, arf, B, d_info, stream)

    def rfp_spfsv_batched(self, batch, d_plan, arf, B, d_info, stream=None):
        return self._batched("rfp_spfsv_batched", batch, d_plan, arf, B, d_info, stream)

    def rfp_ssyrk_tc(self, uplo, n, k, alpha, A, lda, prec, beta, C, ldc, d_err, stream=None):
        rc = self.lib.rfp_ssyrk_tc(_ch(uplo), n, k, alpha, _addr(A), lda, prec, beta, _addr(C), ldc,
                                   _addr(d_err), _stream(stream))
        return self._check("rfp_ssyrk_tc", rc)

    # ---- the rest of the LAPACK 3.2 RFP routine set ----
    def _surface(self, name, args, stream):
        conv = [(_ch(a) if isinstance(a, str) else (_addr(a) if hasattr(a, "data_ptr")
                 or hasattr(a, "ctypes") else a)) for a in args]
        return self._check(name, getattr(self.lib, name)(*conv, _stream(stream)))

    def rfp_dtpttf(self, transr, uplo, n, ap, arf, stream=None):
        return self._surface("rfp_dtpttf", (transr, uplo, n, ap, arf), stream)

    def rfp_stpttf(self, transr, uplo, n, ap, arf, stream=None):
        return self._surface("rfp_stpttf", (transr, uplo, n, ap, arf), stream)

    def rfp_dtfttp(self, transr, uplo, n, arf, ap, stream=None):
        return self._surface("rfp_dtfttp", (transr, uplo, n, arf, ap), stream)

    def rfp_stfttp(self, transr, uplo, n, arf, ap, stream=None):
        return self._surface("rfp_stfttp", (transr, uplo, n, arf, ap), stream)

    def rfp_dtftri(self, transr, uplo, diag, n, arf, info, work=None, stream=None):
        return self._surface("rfp_dtftri", (transr, uplo, diag, n, arf, info, work), stream)

    def rfp_stftri(self, transr, uplo, diag, n, arf, info, work=None, stream=None):
        return self._surface("rfp_stftri", (transr, uplo, diag, n, arf, info, work), stream)

    def rfp_dsfrk(self, transr, uplo, trans, n, k, alpha, A, lda, beta, C, stream=None):
        return self._surface("rfp_dsfrk", (transr, uplo, trans, n, k, alpha, A, lda, beta, C), stream)

    def rfp_ssfrk(self, transr, uplo, trans, n, k, alpha, A, lda, beta, C, stream=None):
        return self._surface("rfp_ssfrk", (transr, uplo, trans, n, k, alpha, A, lda, beta, C), stream)

    def rfp_dtfsm(self, transr, side, uplo, trans, diag, m, n, alpha, arf, B, ldb, stream=None):
        return self._surface("rfp_dtfsm", (transr, side, uplo, trans, diag, m, n, alpha, arf, B, ldb),
                             stream)

    def rfp_stfsm(self, transr, side, uplo, trans, diag, m, n, alpha, arf, B, ldb, stream=None):
        return self._surface("rfp_stfsm", (transr, side, uplo, trans, diag, m, n, alpha, arf, B, ldb),
                             stream)

    def rfp_dlansf(self, norm, transr, uplo, n, arf, work, value, stream=None):
        return self._surface("rfp_dlansf", (norm, transr, uplo, n, arf, work, value), stream)

    def rfp_slansf(self, norm, transr, uplo, n, arf, work, value, stream=None):
        return self._surface("rfp_slansf", (norm, transr, uplo, n, arf, work, value), stream)

    def rfp_dpftrs(self, transr, uplo, n, nrhs, arf, B, ldb, stream=None):
        return self._trs("rfp_dpftrs", transr, uplo, n, nrhs, arf, B, ldb, stream)

    def rfp_spftrs(self, transr, uplo, n, nrhs, arf, B, ldb, stream=None):
        return self._trs("rfp_spftrs", transr, uplo, n, nrhs, arf, B, ldb, stream)


_default = None
_lock = threading.Lock()


def library() -> Library:
    """The CUDA build (loaded once; raises if it has not been built)."""
    global _default
    with _lock:
        if _default is None:
            _default = Library(DEFAULT_LIB)
        return _default


def _fwd(name):
    def f(*args, **kw):
        return getattr(library(), name)(*args, **kw)
    f.__name__ = name
    f.__doc__ = f"Calls the C entry point {name} of include/rfp.h."
    return f


rfp_layout = _fwd("rfp_layout")
rfp_kernel_launches = _fwd("rfp_kernel_launches")
rfp_stage_timing, rfp_stage_times = _fwd("rfp_stage_timing"), _fwd("rfp_stage_times")
rfp_dpack, rfp_spack = _fwd("rfp_dpack"), _fwd("rfp_spack")
rfp_dunpack, rfp_sunpack = _fwd("rfp_dunpack"), _fwd("rfp_sunpack")
rfp_dpftrf, rfp_spftrf = _fwd("rfp_dpftrf"), _fwd("rfp_spftrf")
rfp_dpftrs, rfp_spftrs = _fwd("rfp_dpftrs"), _fwd("rfp_spftrs")
rfp_dpftri, rfp_spftri = _fwd("rfp_dpftri"), _fwd("rfp_spftri")
rfp_ssyrk_tc = _fwd("rfp_ssyrk_tc")
rfp_dpfsv_mixed, rfp_dpfsv_mixed_workspace = _fwd("rfp_dpfsv_mixed"), _fwd("rfp_dpfsv_mixed_workspace")
rfp_dpfsv_mixed_noalloc = _fwd("rfp_dpfsv_mixed_noalloc")
rfp_batch_plan_bytes, rfp_batch_plan = _fwd("rfp_batch_plan_bytes"), _fwd("rfp_batch_plan")
rfp_dpfsv_batched, rfp_spfsv_batched = _fwd("rfp_dpfsv_batched"), _fwd("rfp_spfsv_batched")
rfp_dpfsv_mixed_noalloc_capacity = _fwd("rfp_dpfsv_mixed_noalloc_capacity")
rfp_dtpttf, rfp_stpttf = _fwd("rfp_dtpttf"), _fwd("rfp_stpttf")
rfp_dtfttp, rfp_stfttp = _fwd("rfp_dtfttp"), _fwd("rfp_stfttp")
rfp_dtftri, rfp_stftri = _fwd("rfp_dtftri"), _fwd("rfp_stftri")
rfp_dsfrk, rfp_ssfrk = _fwd("rfp_dsfrk"), _fwd("rfp_ssfrk")
rfp_dtfsm, rfp_stfsm = _fwd("rfp_dtfsm"), _fwd("rfp_stfsm")
rfp_dlansf, rfp_slansf = _fwd("rfp_dlansf"), _fwd("rfp_slansf")
