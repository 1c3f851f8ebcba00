"""Pins for the oracle's RFPF index work (pack / unpack), CPU only.

Each check ties the oracle to something other than itself: the element
placements printed in Figs. 4, 5 and 6, the invariants every layout must
satisfy (a bijection onto n(n+1)/2 slots, unpack(pack(A)) = triangle of A),
and LAPACK's own TRTTF/TFTTR (SciPy), which implement the same format.
"""
import os
import re

import numpy as np
import pytest

import oracle
from rfp_inputs import LAYOUTS

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _coded_matrix(n: int, uplo: str) -> np.ndarray:
    """Full matrix whose UPLO triangle holds a_{i,j} = 100 i + j (1-based)."""
    A = np.full((n, n), -1.0, order="F")
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            if (uplo == "L" and i >= j) or (uplo == "U" and i <= j):
                A[i - 1, j - 1] = 100 * i + j
    return A


def _read_fig6(golden_dir):
    sections, cur = [], None
    with open(os.path.join(golden_dir, "fig6_layouts.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            m = re.match(r"\[N=(\d+) uplo=(\w) transr=(\w) rows=(\d+) cols=(\d+)\]", line)
            if m:
                cur = dict(n=int(m[1]), uplo=m[2], transr=m[3], rows=int(m[4]),
                           cols=int(m[5]), grid=[])
                sections.append(cur)
            else:
                cur["grid"].append([tuple(map(int, t.split(","))) for t in line.split()])
    return sections


def test_fig6_all_eight_layouts(golden_dir):
    secs = _read_fig6(golden_dir)
    assert len(secs) == 8
    assert {(s["n"], s["uplo"], s["transr"]) for s in secs} == {
        (n, u, t) for n in (6, 7) for u in "LU" for t in "NT"}
    for s in secs:
        n = s["n"]
        arf = oracle.pack(s["transr"], s["uplo"], _coded_matrix(n, s["uplo"]))
        assert s["rows"] * s["cols"] == n * (n + 1) // 2 == arf.size
        stored = arf.reshape(s["cols"], s["rows"]).T          # column-major
        expect = np.array([[100 * i + j for (i, j) in row] for row in s["grid"]], float)
        assert expect.shape == stored.shape
        np.testing.assert_array_equal(stored, expect, err_msg=str(s))


def test_fig4_positions_n7_lower(golden_dir):
    rows = np.loadtxt(os.path.join(golden_dir, "fig4_positions_n7.txt"), dtype=int)
    assert len(rows) == 28
    A = _coded_matrix(7, "L")
    flatA = A.ravel(order="F")
    arf = oracle.pack("N", "L", A)
    for i, j, pos_a, pos_ar in rows:
        assert pos_a == i + (j - 1) * 7               # Fig. 1 full format, LDA=7
        assert flatA[pos_a - 1] == 100 * i + j
        assert arf[pos_ar - 1] == 100 * i + j, (i, j, pos_ar)


def test_fig5_fig6_subscripts(golden_dir):
    with open(os.path.join(golden_dir, "fig56_subscripts.txt")) as f:
        rows = [l.split("#")[0].split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for uplo, i, j, pos in rows:
        arf = oracle.pack("N", uplo, _coded_matrix(6, uplo))
        assert arf[int(pos) - 1] == 100 * int(i) + int(j)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 8, 9, 31, 32, 33, 64, 65, 100, 127])
@pytest.mark.parametrize("transr,uplo", LAYOUTS)
def test_bijection_and_roundtrip(n, transr, uplo):
    A = np.asfortranarray(np.arange(1, n * n + 1, dtype=float).reshape(n, n))
    arf = oracle.pack(transr, uplo, A)
    tri = np.tril(A) if uplo == "L" else np.triu(A)
    # every triangle element lands exactly once
    want = np.sort(tri[np.tril_indices(n)] if uplo == "L" else tri[np.triu_indices(n)])
    np.testing.assert_array_equal(np.sort(arf), want)
    # unpack(pack(A)) restores the triangle and leaves the other one alone
    other = np.full((n, n), -7.0, order="F")
    B = oracle.unpack(transr, uplo, n, arf, other)
    mask = np.tril(np.ones((n, n), bool)) if uplo == "L" else np.triu(np.ones((n, n), bool))
    np.testing.assert_array_equal(B[mask], A[mask])
    assert np.all(B[~mask] == -7.0)


def test_small_cases_by_hand():
    # N=1: the array is [a11]; N=2: [a22, a11, a21] lower, [a12, a22, a11] upper
    A = np.array([[11.0, 12.0], [21.0, 22.0]], order="F")
    np.testing.assert_array_equal(oracle.pack("N", "L", A), [22, 11, 21])
    np.testing.assert_array_equal(oracle.pack("N", "U", A), [12, 22, 11])
    np.testing.assert_array_equal(oracle.pack("T", "L", np.array([[5.0]])), [5.0])


@pytest.mark.parametrize("n", [1, 2, 3, 6, 7, 8, 16, 17, 64, 101, 1000, 1001])
@pytest.mark.parametrize("transr,uplo", LAYOUTS)
def test_matches_lapack_trttf_tfttr(n, transr, uplo):
    la = pytest.importorskip("scipy.linalg.lapack")
    rng = np.random.default_rng(n)
    A = np.asfortranarray(rng.standard_normal((n, n)))
    ref, info = la.dtrttf(A, transr=transr, uplo=uplo)
    assert info == 0
    np.testing.assert_array_equal(oracle.pack(transr, uplo, A), ref.ravel(order="F"))
    back, info = la.dtfttr(n, ref, transr=transr, uplo=uplo)
    assert info == 0
    np.testing.assert_array_equal(oracle.unpack(transr, uplo, n, ref),
                                  np.tril(back) if uplo == "L" else np.triu(back))
