"""In-tree build of libmtp.so for sm_103a (GB300).

Steps: run the generator (codegen.py) into csrc/generated/, compile every translation unit with
nvcc in parallel (one -gencode, arch=compute_103a,code=sm_103a), link a shared library into
paper_2007_08555_gb300/_build/libmtp.so.  Objects are rebuilt only when a source is newer.
"""

from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

from . import codegen

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
GEN = os.path.join(CSRC, "generated")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmtp.so")
ROOT = os.path.dirname(HERE)

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", CSRC, "-I", GEN, "-I", os.path.join(ROOT, "include")]

HEADERS = ["mtp_common.cuh", "mtp_level.h", "mtp_level_impl.cuh", "mtp_internal.h", "mtp_gen_common.h"]


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in src_list if os.path.exists(s))


def _compile(args):
    src, obj, deps, verbose = args
    if not _newer([src] + deps, obj):
        return obj, ""
    cmd = [NVCC] + ARCH + FLAGS + ["-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{p.stderr[-8000:]}")
    os.replace(obj + ".tmp", obj)
    return obj, p.stderr


def build(levels=codegen.SUPPORTED_LEVELS, jobs=None, verbose=False) -> str:
    os.makedirs(OUT, exist_ok=True)
    codegen.emit_all(GEN, levels)
    common = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "mtp.h"),
                                                         os.path.join(HERE, "codegen.py")]
    units = []
    for name in ("mtp_api.cu", "mtp_nbr.cu", "mtp_maxvol.cu", "mtp_md.cu", "mtp_peak.cu", "mtp_grade_tc.cu", "mtp_relax.cu", "mtp_train.cu"):
        units.append((os.path.join(CSRC, name), os.path.join(OUT, name.replace(".cu", ".o")), common, verbose))
    for L in levels:
        src = os.path.join(GEN, f"mtp_level_L{L}.cu")
        units.append((src, os.path.join(OUT, f"mtp_level_L{L}.o"), common + [os.path.join(GEN, f"mtp_gen_L{L}.h")],
                      verbose))
    jobs = jobs or min(len(units), max(2, os.cpu_count() or 2))
    # biggest units first so they overlap with the rest
    units.sort(key=lambda u: -os.path.getsize(u[2][-1]) if u[0].endswith(".cu") and "level" in u[0] else 0)
    logs = []
    with ThreadPoolExecutor(jobs) as ex:
        for obj, log in ex.map(_compile, units):
            if log:
                logs.append((obj, log))
    objs = [u[1] for u in units]
    if _newer(objs, LIB):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcudart"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed:\n{p.stderr[-8000:]}")
        os.replace(LIB + ".tmp", LIB)
    if verbose:
        for obj, log in logs:
            sys.stderr.write(f"== {obj}\n{log}\n")
    return LIB


if __name__ == "__main__":
    import time

    t = time.time()
    print(build(verbose="-v" in sys.argv), f"{time.time() - t:.1f}s")
