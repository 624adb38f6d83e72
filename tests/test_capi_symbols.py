"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/flinng.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "flinng.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(flinng_[a-z_0-9]+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_five_entry_points():
    syms = declared_symbols()
    for s in ("flinng_create", "flinng_build", "flinng_insert", "flinng_query", "flinng_destroy"):
        assert s in syms


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_builds_loads_and_exports_all_symbols():
    from paper_2106_11565_gb300 import _build, flinng
    path = _build.build()
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    # the binding knows every declared symbol with a signature
    assert set(declared_symbols()) == set(flinng._SIGS)
    # last_error needs no device
    flinng._lib = None
    assert flinng.load().flinng_last_error() == b""
    assert flinng.load().flinng_destroy(None) == 0
