"""Model files (mtp_save / mtp_load) on the host: every malformed file is refused with MTP_EINVAL
before any device work, and the handle stays NULL.  No GPU: mtp_load reads and checks the whole
file first, and none of these files passes the check."""

import ctypes
import os

import numpy as np
import pytest

from paper_2007_08555_gb300 import mtp

EINVAL = 1


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(mtp.LIB_PATH):
        from paper_2007_08555_gb300 import build

        build.build()
    return mtp.load()


def _text(lev=10, S=1, NQ=2, m=17, nmu=3, xi=None, c=None, version=1, magic="mtp-gb300-potential",
          precision="fp32", lanes="0 0", active=None, tail="end\n"):
    xi = np.linspace(-1, 1, m) if xi is None else xi
    c = np.linspace(0.1, 0.6, S * S * nmu * NQ) if c is None else c
    out = [f"{magic} {version}", f"lev_max {lev}", f"n_species {S}", f"n_radial {NQ}", "r_min 2", "r_cut 5",
           f"precision {precision}", "skin 0.5", "neighbor_capacity 96", f"threads_per_atom {lanes}",
           f"xi {len(xi)}", " ".join(repr(float(v)) if isinstance(v, (float, np.floating)) else str(v) for v in xi),
           f"c {len(c)}", " ".join(repr(float(v)) if isinstance(v, (float, np.floating)) else str(v) for v in c)]
    out += active if active is not None else ["active_set 0"]
    return "\n".join(out) + "\n" + tail


def _load(lib, tmp_path, text):
    p = tmp_path / "model.txt"
    p.write_text(text)
    h = ctypes.c_void_p(12345)
    code = lib.mtp_load(os.fsencode(str(p)), ctypes.byref(h))
    return code, h.value


def test_missing_file(lib, tmp_path):
    h = ctypes.c_void_p(12345)
    assert lib.mtp_load(os.fsencode(str(tmp_path / "absent.txt")), ctypes.byref(h)) == EINVAL
    assert h.value is None


@pytest.mark.parametrize("case", [
    dict(magic="mtp-potential"),
    dict(version=3),
    dict(version=2),                                    # version 2 needs the grade_kind record
    dict(version=2, active=["grade_kind 2", "active_set 0"]),
    dict(version=2, active=["grade_kind 1 3", "0 5 5", "active_set 0"]),   # columns must ascend
    dict(version=2, active=["grade_kind 1 2", "0 23", "active_set 0"]),    # m + #c = 23 columns
    dict(version=2, active=["grade_kind 1 2", "0 1", "active_set 1", "A 9", "1 0 0 1"]),
    dict(lev=11),
    dict(lev=22),
    dict(S=9),
    dict(NQ=0),
    dict(precision="fp16"),
    dict(lanes="3 0"),
    dict(xi=np.zeros(16)),                              # lev 10 has m = 17
    dict(c=np.zeros(5)),                                # S * S * N_mu * N_Q = 6
    dict(xi=[0.0] * 16 + ["nan"]),
    dict(xi=[0.0] * 16 + ["1e400"]),
    dict(c=[0.0] * 5 + ["0x"]),
    dict(tail=""),                                      # no end marker
    dict(tail="end\n1.0\n"),                            # data after the end marker
    dict(active=["active_set 2"]),
    dict(active=["active_set 1", "A 3", "1 2 3"]),       # A needs m * m values
])
def test_malformed_file_is_refused(lib, tmp_path, case):
    code, h = _load(lib, tmp_path, _text(**case))
    assert code == EINVAL
    assert h is None


def test_r_min_not_below_r_cut_is_refused(lib, tmp_path):
    text = _text().replace("r_min 2", "r_min 5")
    assert _load(lib, tmp_path, text) == (EINVAL, None)


def test_truncated_values_are_refused(lib, tmp_path):
    text = _text()
    cut = text.index("\nc ")
    assert _load(lib, tmp_path, text[:cut - 3]) == (EINVAL, None)
