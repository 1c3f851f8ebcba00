"""Planted mistakes: each one is put into a copy of the oracle's C source, on
the CPU, and the pin tests must reject the copy.  This shows the pins are
strong enough that a dropped term, a wrong sign or index, a transposed operand
or a wrong offset anywhere in the oracle would be caught."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rfp_oracle.c")

MUTANTS = {
    "chol_dropped_term": ("for (int64_t p = 0; p < j; ++p) t -= S[i * n + p] * S[j * n + p];",
                          "for (int64_t p = 0; p + 1 < j; ++p) t -= S[i * n + p] * S[j * n + p];"),
    "chol_wrong_op": ("S[i * n + j] = t / ljj;", "S[i * n + j] = t * ljj;"),
    "chol_zero_pivot_accepted": ("if (!(s > 0.0)) return", "if (s < 0.0) return"),
    "pack_lower_odd_transposed": ("MOVE(r, c + 1, n1 + c, n1 + r)", "MOVE(r, c + 1, n1 + r, n1 + c)"),
    "pack_lower_even_offset": ("MOVE(1 + i, j, i, j)", "MOVE(i + (i == j), j, i, j)"),
    "pack_upper_offset": ("MOVE(n1 + 1 + r, c, c, r)", "MOVE(n1 + 1 + r, c, r, c)"),
    "pack_transr_index": ("if (is_trans(transr)) arf[c + r * nc]", "if (is_trans(transr)) arf[r + c * nc]"),
    "solve_back_transposed": ("t -= L[p * n + i] * b[p];", "t -= L[i * n + p] * b[p];"),
    "solve_fwd_sign": ("for (int64_t p = 0; p < i; ++p) t -= L[i * n + p] * b[p];",
                       "for (int64_t p = 0; p < i; ++p) t += L[i * n + p] * b[p];"),
    "inv_dropped_term": ("for (int64_t k = i; k < n; ++k) t +=", "for (int64_t k = i + 1; k < n; ++k) t +="),
    "inv_identity_rhs": ("double t = (i == c) ? 1.0 : 0.0;", "double t = 1.0;"),
    "residual_dropped_diag": ("for (int64_t p = 0; p <= c; ++p)", "for (int64_t p = 0; p < c; ++p)"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                    "-shared", str(path), "-o", str(so), "-lm"], check=True)
    return so


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistake(tmp_path, name):
    old, new = MUTANTS[name]
    so = _build_mutant(tmp_path, name, old, new)
    env = dict(os.environ, RFP_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_layout_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_numerics_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout or "Error" in r.stdout
