"""The C-ABI library loads and exports every function declared in include/mtp.h (no GPU calls)."""

import ctypes
import os

import pytest

from paper_2007_08555_gb300 import mtp


@pytest.fixture(scope="module")
def built_lib():
    if not os.path.exists(mtp.LIB_PATH):
        from paper_2007_08555_gb300 import build

        build.build()
    return ctypes.CDLL(mtp.LIB_PATH)


def test_library_exports_every_declared_function(built_lib):
    names = mtp.header_functions()
    assert "mtp_create" in names and "mtp_eval_batch" in names and len(names) >= 15
    missing = [n for n in names if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    # every declared function has a marshalling signature in the Python binding
    names = set(mtp.header_functions())
    assert names <= set(mtp._SIGS), sorted(names - set(mtp._SIGS))


def test_status_strings(built_lib):
    built_lib.mtp_status_str.restype = ctypes.c_char_p
    assert built_lib.mtp_status_str(0) == b"ok"
    assert built_lib.mtp_status_str(4) == b"neighbour list capacity exceeded"
