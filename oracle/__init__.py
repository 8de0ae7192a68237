"""FP64 CPU oracle of the Moment Tensor Potential hot path (Sec. 2.1-2.3).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg may import this package.  The product library never links, loads or calls it, and it shares
no code with the CUDA path: its basis enumeration (levels.py), its evaluation (mtp_oracle.cpp),
its MaxVol (maxvol.py) and its loss (loss.py) are written separately from the definitions.

The C++ part is compiled on first use (or by build()) into oracle/_build/liboracle.so.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import levels

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mtp_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain g++, -O2, no FMA contraction, OpenMP)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.oracle_model_create.restype = P
            L.oracle_model_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, ip, ctypes.c_int]
            L.oracle_model_free.argtypes = [P]
            L.oracle_model_nmu.argtypes = [P]
            L.oracle_model_m.argtypes = [P]
            L.oracle_radial.argtypes = [P, ctypes.c_double, dp, dp]
            L.oracle_neighbors.restype = ctypes.c_long
            L.oracle_neighbors.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ip, ctypes.c_int, ip, ip, ip,
                                           dp, ctypes.c_long]
            L.oracle_eval.restype = ctypes.c_int
            L.oracle_eval.argtypes = [P, dp, dp, ctypes.c_int, dp, ip, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp,
                                      dp, ctypes.c_int]
            L.oracle_eval_sampled.restype = ctypes.c_int
            L.oracle_eval_sampled.argtypes = [P, dp, dp, ctypes.c_int, dp, ip, dp, ip, ctypes.c_int, dp, dp, dp,
                                              ctypes.c_int]
            _lib = L
    return _lib


def _d(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def neighbors(pos, cell, r_cut, which=None):
    """Canonical neighbour lists (Eq. 1): per listed atom, every (j, s) with |x_j + s H - x_i| < R_cut,
    sorted by (j, s).  Returns (counts [k], j [P], s [P,3], r_ij [P,3])."""
    pos, cell = _f64(pos), _f64(cell)
    n = pos.shape[0]
    w = None if which is None else _i32(which)
    k = n if w is None else w.shape[0]
    counts = np.zeros(k, dtype=np.int32)
    total = lib().oracle_neighbors(n, _d(pos), _d(cell), float(r_cut), _i(w), k, _i(counts), None, None, None, 0)
    j = np.zeros(total, dtype=np.int32)
    s = np.zeros((total, 3), dtype=np.int32)
    d = np.zeros((total, 3), dtype=np.float64)
    got = lib().oracle_neighbors(n, _d(pos), _d(cell), float(r_cut), _i(w), k, _i(counts), _i(j), _i(s), _d(d),
                                 total)
    assert got == total
    return counts, j, s, d


class Potential:
    """The oracle's view of one potential: its own level table plus theta = {xi, c}."""

    def __init__(self, params):
        self.p = params
        self.table = np.asarray(levels.level_table(params.lev_max), dtype=np.int32)
        self.h = lib().oracle_model_create(params.lev_max, params.n_species, params.n_radial, params.r_min,
                                           params.r_cut, _i(self.table), self.table.shape[0])
        self.m = lib().oracle_model_m(self.h)
        self.n_mu = lib().oracle_model_nmu(self.h)
        assert self.m == len(params.xi), (self.m, len(params.xi))
        assert params.c.shape == (params.n_species, params.n_species, self.n_mu, params.n_radial)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.oracle_model_free(self.h)
            self.h = None

    def eval(self, cfg, xi=None, c=None, dxi=None, dc=None, want_b=False, threads=0):
        """E, F [n,3], W [3,3] (W = -dE/d eps), site energies [n] and optionally per-atom B [n,m];
        with tangents (dxi, dc) also their exact derivatives along that direction of theta."""
        xi = _f64(self.p.xi if xi is None else xi)
        c = _f64(self.p.c if c is None else c)
        pos, types, cell = _f64(cfg.pos), _i32(cfg.types), _f64(cfg.cell)
        n = pos.shape[0]
        e = np.zeros(1)
        f = np.zeros((n, 3))
        w = np.zeros(9)
        site = np.zeros(n)
        b = np.zeros((n, self.m)) if want_b else None
        tang = dxi is not None
        de = np.zeros(1) if tang else None
        dfo = np.zeros((n, 3)) if tang else None
        dw = np.zeros(9) if tang else None
        dxi = _f64(dxi) if tang else None
        dc = _f64(dc) if tang else None
        rc = lib().oracle_eval(self.h, _d(xi), _d(c), n, _d(pos), _i(types), _d(cell), _d(e), _d(f), _d(w), _d(site),
                               _d(b), _d(dxi), _d(dc), _d(de), _d(dfo), _d(dw), int(threads))
        if rc != 0:
            raise ValueError("oracle_eval: species index out of range")
        out = {"energy": float(e[0]), "forces": f, "virial": w.reshape(3, 3), "site": site}
        if want_b:
            out["b_atoms"] = b
        if tang:
            out["d_energy"] = float(de[0])
            out["d_forces"] = dfo
            out["d_virial"] = dw.reshape(3, 3)
        return out

    def radial_basis(self, r):
        """(Q_b(r), dQ_b/dr) for b = 1..N_Q (Eq. 4), r < R_cut."""
        q = np.zeros(self.p.n_radial)
        dq = np.zeros(self.p.n_radial)
        lib().oracle_radial(self.h, float(r), _d(q), _d(dq))
        return q, dq

    def eval_sampled(self, cfg, which, threads=0):
        """Site energies, basis rows and forces of the listed atoms only (for large cells): V_i, B(n_i)
        and F_i = -dE/dx_i, with the neighbour lists searched among the atoms within 2 R_cut."""
        which = _i32(which)
        pos, types, cell = _f64(cfg.pos), _i32(cfg.types), _f64(cfg.cell)
        k = which.shape[0]
        site = np.zeros(k)
        b = np.zeros((k, self.m))
        f = np.zeros((k, 3))
        rc = lib().oracle_eval_sampled(self.h, _d(_f64(self.p.xi)), _d(_f64(self.p.c)), pos.shape[0], _d(pos),
                                       _i(types), _d(cell), _i(which), k, _d(site), _d(b), _d(f), int(threads))
        if rc != 0:
            raise ValueError("oracle_eval_sampled: atom or species index out of range")
        return {"site": site, "b_atoms": b, "forces": f}
