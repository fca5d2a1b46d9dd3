"""The C ABI library loads and exports everything include/sa.h declares.
No GPU: only calls that are rejected on the host before any CUDA work."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "sa.h")


@pytest.fixture(scope="module")
def salib():
    from paper_1303_3692_gb300 import build_lib, sa

    build_lib.build()
    return sa


def declared_functions():
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sa_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sa_build", "sa_search_batch", "sa_locate", "sa_free", "sa_strerror", "sa_save", "sa_load",
                     "sa_index_info"):
        assert required in names


def test_every_declared_symbol_is_exported(salib):
    lib = ctypes.CDLL(salib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(salib.SIGNATURES)


def test_strerror_and_version(salib):
    assert salib.sa_strerror(0) == "success"
    for code in range(-8, 0):
        assert salib.sa_strerror(code) != "unknown status"
    assert salib.sa_strerror(-99) == "unknown status"
    assert salib.lib().sa_version() == 0x000100


def test_host_side_argument_checks(salib):
    L = salib.lib()
    h = ctypes.c_void_p()
    assert L.sa_build(None, 10, salib.SA_W32, None, ctypes.byref(h)) == salib.SA_ERR_ARG
    buf = ctypes.create_string_buffer(b"ACGT")
    assert L.sa_build(ctypes.cast(buf, ctypes.c_void_p), 0, salib.SA_W32, None, ctypes.byref(h)) == salib.SA_ERR_ARG
    assert L.sa_build(ctypes.cast(buf, ctypes.c_void_p), 4, 0, None, ctypes.byref(h)) == salib.SA_ERR_ARG
    assert L.sa_build(ctypes.cast(buf, ctypes.c_void_p), 4, 3, None, ctypes.byref(h)) == salib.SA_ERR_ARG
    assert L.sa_search_batch(None, 1, None, None, None, 1, None, None) == salib.SA_ERR_ARG
    assert L.sa_locate(None, 1, None, None, 1, 4, None, None, 0, None) == salib.SA_ERR_ARG
    assert L.sa_index_info(None, None, None, None, None, None) == salib.SA_ERR_ARG
    assert L.sa_copy_kmer_table(None, None, None) == salib.SA_ERR_ARG
    assert L.sa_save(None, b"/nonexistent", None) == salib.SA_ERR_ARG
    L.sa_free(None)


def test_result_struct_layout(salib):
    assert ctypes.sizeof(salib.sa_result) == 32  # one DRAM sector per result
    assert ctypes.sizeof(salib.sa_search_params) == 72
