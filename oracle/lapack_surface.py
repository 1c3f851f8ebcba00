"""Oracle of the rest of the LAPACK 3.2 RFP routine set (test infrastructure
only, like the rest of this package).

The paper's table of the new LAPACK routines (Table lapack) lists, besides
PFTRF / PFTRS / PFTRI and the full-format conversions TRTTF / TFTTR:
TPTTF / TFTTP (standard packed <-> RFP), TFTRI (triangular inverse in RFP),
SFRK (symmetric rank-k update of an RFP matrix), TFSM (triangular solve with
an RFP triangle) and LANSF (norm of a symmetric RFP matrix).  Each function
below is that routine's definition written out on full matrices: the RFP
array is expanded with this package's own ``unpack``, the operation is done
in FP64 with plain loops or a numpy primitive, and the result is packed back
with ``pack``.  No blocking, no reordering beyond the definition.

Packed storage (TP), column-major, 0-based:
  UPLO = 'U': AP[i + j (j + 1) / 2] = A(i, j) for 0 <= i <= j < n
  UPLO = 'L': AP[i + j (2n - j - 1) / 2] = A(i, j) for 0 <= j <= i < n
"""
from __future__ import annotations

import numpy as np

from .oracle import pack, unpack


def _lower(uplo: str) -> bool:
    return uplo.upper() == "L"


def tp_index(uplo: str, n: int, i: int, j: int) -> int:
    """Position of A(i, j) (in the UPLO triangle) in the packed array."""
    if _lower(uplo):
        assert i >= j
        return i + j * (2 * n - j - 1) // 2
    assert i <= j
    return i + j * (j + 1) // 2


def tp_to_full(uplo: str, n: int, ap) -> np.ndarray:
    """Full n x n matrix holding the UPLO triangle of a packed array (zeros elsewhere)."""
    A = np.zeros((n, n), order="F")
    for j in range(n):
        rows = range(j, n) if _lower(uplo) else range(0, j + 1)
        for i in rows:
            A[i, j] = ap[tp_index(uplo, n, i, j)]
    return A


def full_to_tp(uplo: str, A) -> np.ndarray:
    n = A.shape[0]
    ap = np.zeros(n * (n + 1) // 2)
    for j in range(n):
        rows = range(j, n) if _lower(uplo) else range(0, j + 1)
        for i in rows:
            ap[tp_index(uplo, n, i, j)] = A[i, j]
    return ap


def tpttf(transr: str, uplo: str, n: int, ap) -> np.ndarray:
    """TPTTF: the packed triangle in RFP (Table lapack)."""
    return pack(transr, uplo, tp_to_full(uplo, n, ap))


def tfttp(transr: str, uplo: str, n: int, arf) -> np.ndarray:
    """TFTTP: the RFP triangle in packed storage (Table lapack)."""
    return full_to_tp(uplo, unpack(transr, uplo, n, arf))


def _triangle(transr, uplo, n, arf, unit):
    T = unpack(transr, uplo, n, arf)
    T = np.tril(T) if _lower(uplo) else np.triu(T)
    if unit:
        np.fill_diagonal(T, 1.0)
    return T


def tri_inverse(T, lower: bool) -> np.ndarray:
    """Inverse of a triangular matrix, column by column: W e_c solves T w = e_c
    by substitution in the triangle's own order."""
    n = T.shape[0]
    W = np.zeros((n, n), order="F")
    for c in range(n):
        w = np.zeros(n)
        order = range(n) if lower else range(n - 1, -1, -1)
        for i in order:
            if lower:
                s = (1.0 if i == c else 0.0) - T[i, :i] @ w[:i]
            else:
                s = (1.0 if i == c else 0.0) - T[i, i + 1:] @ w[i + 1:]
            w[i] = s / T[i, i]
        W[:, c] = w
    return W


def tftri(transr: str, uplo: str, diag: str, n: int, arf):
    """TFTRI (Table lapack): the inverse of the RFP triangle, in place.
    Returns (arf_inv, info); info = first zero diagonal (1-based) when DIAG =
    'N'.  With DIAG = 'U' the diagonal is taken as 1, is not referenced and
    comes back unchanged."""
    unit = diag.upper() == "U"
    T = _triangle(transr, uplo, n, arf, unit)
    if not unit:
        zero = np.nonzero(np.diag(T) == 0.0)[0]
        if zero.size:
            return np.array(arf, dtype=np.float64, copy=True), int(zero[0]) + 1
    W = tri_inverse(T, _lower(uplo))
    if unit:   # keep the stored (unreferenced) diagonal
        stored = np.diag(unpack(transr, uplo, n, arf))
        np.fill_diagonal(W, stored)
    return pack(transr, uplo, W), 0


def sfrk(transr: str, uplo: str, trans: str, n: int, k: int, alpha: float, A, beta: float, arf):
    """SFRK (Table lapack): C := alpha op(A) op(A)^T + beta C, C symmetric in
    RFP (its UPLO triangle), op(A) = A (n x k, TRANS = 'N') or A^T (A k x n,
    TRANS = 'T').  beta = 0: C is not read."""
    opA = np.asarray(A, dtype=np.float64)
    opA = opA if trans.upper() == "N" else opA.T
    assert opA.shape == (n, k)
    if beta == 0.0:
        C = np.zeros((n, n))
    else:
        C = unpack(transr, uplo, n, arf)
        C = np.tril(C) + np.tril(C, -1).T if _lower(uplo) else np.triu(C) + np.triu(C, 1).T
    R = alpha * (opA @ opA.T) + beta * C
    return pack(transr, uplo, R)


def tfsm(transr: str, side: str, uplo: str, trans: str, diag: str, m: int, nc: int, alpha: float,
         arf, B) -> np.ndarray:
    """TFSM (Table lapack): B := alpha op(A)^{-1} B (SIDE = 'L', A of order m)
    or alpha B op(A)^{-1} (SIDE = 'R', A of order nc); A triangular in RFP,
    op(A) = A or A^T, unit diagonal when DIAG = 'U'.  alpha = 0: B := 0."""
    B = np.array(B, dtype=np.float64, order="F", copy=True)
    assert B.shape == (m, nc)
    if alpha == 0.0:
        return np.zeros_like(B)
    left = side.upper() == "L"
    order = m if left else nc
    T = _triangle(transr, uplo, order, arf, diag.upper() == "U")
    notrans = trans.upper() == "N"
    opA = T if notrans else T.T
    Winv = tri_inverse(opA, _lower(uplo) == notrans)   # op(A) lower: (L, N) or (U, T)
    return alpha * (Winv @ B) if left else alpha * (B @ Winv)


def lansf(norm: str, transr: str, uplo: str, n: int, arf) -> float:
    """LANSF (Table lapack): 'M' max |a_ij|, '1' / 'O' / 'I' one / infinity
    norm (equal for a symmetric matrix), 'F' / 'E' Frobenius norm, of the
    symmetric matrix whose UPLO triangle is in RFP."""
    if n == 0:
        return 0.0
    C = unpack(transr, uplo, n, arf)
    A = np.tril(C) + np.tril(C, -1).T if _lower(uplo) else np.triu(C) + np.triu(C, 1).T
    key = norm.upper()
    if key == "M":
        return float(np.max(np.abs(A)))
    if key in ("1", "O", "I"):
        return float(np.max(np.sum(np.abs(A), axis=0)))
    if key in ("F", "E"):
        return float(np.sqrt(np.sum(A * A)))
    raise ValueError(norm)
