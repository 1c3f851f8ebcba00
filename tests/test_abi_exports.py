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
