"""The C-ABI library loads and exports every entry point of include/hcc.h (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hcc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(hcc_[a-z_0-9]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_16652_gb300 import build, hcc
    build()
    return hcc.load()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for f in ("hcc_select_cut", "hcc_encode", "hcc_sort", "hcc_gather", "hcc_trace", "hcc_run", "hcc_run_host",
              "hcc_create", "hcc_destroy", "hcc_sync", "hcc_bvh_upload"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_status_strings_need_no_gpu(lib):
    lib.hcc_status_string.restype = ctypes.c_char_p
    assert lib.hcc_status_string(0) == b"HCC_OK"
    assert lib.hcc_status_string(5) == b"HCC_ERR_STACK_OVERFLOW"


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2305_16652_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".c", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
                assert "hcc_oracle" not in text and "libhcc_oracle" not in text, f


def test_binding_declares_every_entry_point(lib):
    """Every function of the header has an explicit ctypes signature in the binding."""
    from paper_2305_16652_gb300 import hcc
    for f in declared_functions():
        assert getattr(lib, f).argtypes is not None or f in ("hcc_last_error", "hcc_status_string"), f
        assert hasattr(hcc, f) or f in ("hcc_last_error", "hcc_status_string"), f
