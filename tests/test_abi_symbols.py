"""The C-ABI library builds for sm_103a, loads, and exports every function include/pcexp.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pcexp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(pcexp_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["pcexp_create", "pcexp_destroy", "pcexp_residual", "pcexp_jvp", "pcexp_step",
              "pcexp_arnoldi", "pcexp_phi", "pcexp_march_steady", "pcexp_status_string"]:
        assert n in names


def test_library_loads_and_exports_every_symbol():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit to build the library")
    from paper_1801_06300_gb300 import build
    path = build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1801_06300_gb300 import capi
    assert set(capi.SIGNATURES) == set(declared_functions())
    lib.pcexp_status_string.restype = ctypes.c_char_p
    assert lib.pcexp_status_string(-2) == b"invalid mesh"
