"""The CUDA library loads on a machine without a GPU and exports every
function declared in include/*.h (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

from paper_0901_1696_gb300 import build as gpu_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(rfp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["rfp_dpack", "rfp_dunpack", "rfp_dpftrf", "rfp_dpftrs", "rfp_dpftri",
                     "rfp_spack", "rfp_sunpack", "rfp_spftrf", "rfp_spftrs", "rfp_spftri",
                     "rfp_layout", "rfp_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    path = gpu_build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_without_gpu():
    from paper_0901_1696_gb300.binding import Library, RfpError
    lib = Library(gpu_build.build())
    d = lib.rfp_layout("N", "L", 7)
    assert (d["n1"], d["n2"], d["ld"], d["t2_off"], d["t2_trans"]) == (4, 3, 7, 7, 1)
    with pytest.raises(RfpError) as e:
        lib.rfp_dpftrf("Q", "L", 7, 0, 0, 0)
    assert e.value.status == -1
    assert lib.lib.rfp_status_string(-3).decode().startswith("invalid argument")


def test_batch_plan_validation_without_gpu():
    """rfp_batch_plan rejects an invalid entry on the host, before any CUDA
    call, and names it."""
    import numpy as np
    from paper_0901_1696_gb300.binding import Library, RfpError, batch_entry_dtype
    lib = Library(gpu_build.build())
    e = np.zeros(3, dtype=batch_entry_dtype())
    e["transr"], e["uplo"], e["n"], e["nrhs"] = b"N", b"L", 10, 0
    e["arf"] = [0, 55, 110]
    fake_plan = 1 << 20                      # 256-byte aligned address, never touched
    for k, field, value in [(1, "n", 513), (2, "arf", 120), (0, "transr", b"C"), (1, "nb", 8),
                            (2, "nrhs", 9)]:
        bad = e.copy()
        bad[field][k] = value
        with pytest.raises(RfpError) as err:
            lib.rfp_batch_plan(3, bad, 165, 0, fake_plan, lib.rfp_batch_plan_bytes(3), 0)
        assert err.value.status == -2 and f"entry {k}" in str(err.value)
    rhs = e.copy()
    rhs["nrhs"][0], rhs["ldb"][0], rhs["b"][0] = 2, 10, 5       # needs 5 + 10 + 10 = 25 > 20
    with pytest.raises(RfpError) as err:
        lib.rfp_batch_plan(3, rhs, 165, 20, fake_plan, lib.rfp_batch_plan_bytes(3), 0)
    assert "entry 0" in str(err.value)
    assert batch_entry_dtype().itemsize == 40
