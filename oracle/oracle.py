"""ctypes front end of the C oracle (``rfp_oracle.c``), numpy in and out.

Test infrastructure only: see the package docstring.  Matrices are numpy
float64 arrays; full matrices are handled column-major (Fortran order) as in
LAPACK.  Every function returns new arrays and leaves its inputs untouched.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rfp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_NAME = "liboracle.so"
_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    pass


def lib_path() -> str:
    return os.path.join(_OUT_DIR, _LIB_NAME)


def build(force: bool = False) -> str:
    """Compile ``rfp_oracle.c`` with gcc into ``oracle/_build/liboracle.so``.

    -ffp-contract=off keeps every multiply-add as two roundings, as written.
    """
    out = lib_path()
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # A planted-mistake copy of the oracle may be substituted by the
        # mutation tests (tests/test_oracle_mutants.py) through this variable.
        lib = ctypes.CDLL(os.environ.get("RFP_ORACLE_LIB") or build())
        i64, c, dp, d = ctypes.c_int64, ctypes.c_char, ctypes.c_void_p, ctypes.c_double
        sig = {
            "oracle_pack": (ctypes.c_int, [c, c, i64, dp, i64, dp]),
            "oracle_unpack": (ctypes.c_int, [c, c, i64, dp, dp, i64]),
            "oracle_potrf_rowmajor": (ctypes.c_int, [i64, dp]),
            "oracle_pftrf": (ctypes.c_int, [c, c, i64, dp]),
            "oracle_pftrs": (ctypes.c_int, [c, c, i64, i64, dp, dp, i64]),
            "oracle_pftri": (ctypes.c_int, [c, c, i64, dp]),
            "oracle_factor_residual": (d, [i64, dp, i64, dp, i64]),
            "oracle_solve_backward_error": (d, [i64, i64, dp, i64, dp, i64, dp, i64]),
            "oracle_inverse_residual": (d, [i64, dp, i64, dp, i64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _ch(x: str) -> bytes:
    return x.encode()[:1]


def ar_shape(n: int):
    """(LDAR, nc) of A_R: LDAR = N (odd) or N+1 (even), nc = ceil(N/2)."""
    return (n if n % 2 else n + 1), (n + 1) // 2


def split(uplo: str, n: int):
    """Block split (n1, n2) of the logical lower factor, as drawn in Figs. 4-6:
    lower layouts put ceil(N/2) rows in A11, upper layouts floor(N/2)."""
    n1 = (n + 1) // 2 if uplo.upper() == "L" else n // 2
    return n1, n - n1


def _f64_fortran(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="F", copy=True)


def pack(transr: str, uplo: str, A) -> np.ndarray:
    """TRTTF: the UPLO triangle of full A (n x n) -> RFP array of n(n+1)/2."""
    A = _f64_fortran(A)
    n = A.shape[0]
    arf = np.zeros(n * (n + 1) // 2, dtype=np.float64)
    if n:
        rc = _load().oracle_pack(_ch(transr), _ch(uplo), n, _ptr(A), n, _ptr(arf))
        if rc:
            raise OracleError("oracle_pack failed")
    return arf


def unpack(transr: str, uplo: str, n: int, arf, A=None) -> np.ndarray:
    """TFTTR: RFP array -> UPLO triangle of a full matrix.  The other triangle
    is taken from ``A`` (zeros if None) and left as it was."""
    arf = np.ascontiguousarray(arf, dtype=np.float64)
    assert arf.size == n * (n + 1) // 2
    out = _f64_fortran(A) if A is not None else np.zeros((n, n), order="F")
    if n:
        rc = _load().oracle_unpack(_ch(transr), _ch(uplo), n, _ptr(arf), _ptr(out), n)
        if rc:
            raise OracleError("oracle_unpack failed")
    return out


def potrf_full(A):
    """Textbook Cholesky of a full symmetric matrix (lower triangle read).
    Returns (L, info) with L lower triangular (upper part zero)."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    S = np.ascontiguousarray(np.tril(A) + np.tril(A, -1).T)   # row-major
    info = _load().oracle_potrf_rowmajor(n, _ptr(S)) if n else 0
    return np.tril(S), int(info)


def pftrf(transr: str, uplo: str, n: int, arf):
    """PFTRF: returns (factor in the same RFP layout, info)."""
    out = np.array(arf, dtype=np.float64, copy=True)
    info = _load().oracle_pftrf(_ch(transr), _ch(uplo), n, _ptr(out)) if n else 0
    if info < 0:
        raise OracleError("oracle_pftrf allocation failure")
    return out, int(info)


def pftrs(transr: str, uplo: str, n: int, arf, B) -> np.ndarray:
    """PFTRS: returns X with A X = B, A's factor in ``arf``."""
    arf = np.ascontiguousarray(arf, dtype=np.float64)
    X = _f64_fortran(B)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    nrhs = X.shape[1]
    if n and nrhs:
        rc = _load().oracle_pftrs(_ch(transr), _ch(uplo), n, nrhs, _ptr(arf), _ptr(X), n)
        if rc:
            raise OracleError("oracle_pftrs failed")
    return X


def pftri(transr: str, uplo: str, n: int, arf):
    """PFTRI: returns (UPLO triangle of A^{-1} in the same layout, info)."""
    out = np.array(arf, dtype=np.float64, copy=True)
    info = _load().oracle_pftri(_ch(transr), _ch(uplo), n, _ptr(out)) if n else 0
    if info < 0:
        raise OracleError("oracle_pftri allocation failure")
    return out, int(info)


def factor_residual(A, L) -> float:
    """||A - L L^T||_F / ||A||_F (compensated inner products)."""
    A, L = _f64_fortran(A), _f64_fortran(L)
    n = A.shape[0]
    return float(_load().oracle_factor_residual(n, _ptr(A), n, _ptr(L), n)) if n else 0.0


def solve_backward_error(A, X, B) -> float:
    """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    A, X, B = _f64_fortran(A), _f64_fortran(X), _f64_fortran(B)
    if X.ndim == 1:
        X, B = X.reshape(-1, 1, order="F"), B.reshape(-1, 1, order="F")
    n, nrhs = X.shape
    if not n or not nrhs:
        return 0.0
    return float(_load().oracle_solve_backward_error(n, nrhs, _ptr(A), n, _ptr(X), n,
                                                     _ptr(B), n))


def inverse_residual(A, X) -> float:
    """||A X - I||_1 / (||A||_1 ||X||_1) (compensated inner products)."""
    A, X = _f64_fortran(A), _f64_fortran(X)
    n = A.shape[0]
    return float(_load().oracle_inverse_residual(n, _ptr(A), n, _ptr(X), n)) if n else 0.0
