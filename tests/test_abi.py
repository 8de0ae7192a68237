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


def test_plain_c_program_links_and_calls(built_lib, tmp_path):
    """The header is plain C99: a C program compiles against it, links libmtp.so and calls entry
    points that need no GPU (status strings, argument checks, refusal of a malformed model file)."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    bad = tmp_path / "bad.txt"
    bad.write_text("not a model\n")
    src = tmp_path / "use_mtp.c"
    src.write_text(f"""
#include <stdio.h>
#include <string.h>
#include "mtp.h"
int main(void) {{
    mtp_model* m = (mtp_model*)1;
    if (strcmp(mtp_status_str(MTP_EOVERFLOW), "neighbour list capacity exceeded") != 0) return 1;
    if (mtp_load("{bad}", &m) != MTP_EINVAL || m != NULL) return 2;
    if (mtp_create(3, 1, 4, 2.0, 5.0, NULL, NULL, MTP_FP64, NULL) != MTP_EINVAL) return 3;
    if (mtp_basis_count(NULL) != 0) return 4;
    if (mtp_set_skin(NULL, 0.1) != MTP_EINVAL) return 5;
    mtp_destroy(NULL);
    printf("ok\\n");
    return 0;
}}
""")
    exe = tmp_path / "use_mtp"
    libdir = os.path.dirname(mtp.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"), str(src), "-o",
                    str(exe), "-L", libdir, "-lmtp", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)
