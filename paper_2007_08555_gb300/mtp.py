"""Python binding of libmtp.so (the C ABI declared in include/mtp.h).

Argument marshalling only: every step of the computation runs in the library's CUDA kernels.
torch provides device memory and streams.  The library is loaded from the package's in-tree
build directory; if it is missing the import of this module still works but load() raises, so a
GPU run can never fall back to another implementation.
"""

from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmtp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mtp.h")

FP64, FP32, FP32_TC = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp32_tc": FP32_TC}
HOST_MEMORY, ASYNC, REUSE_NEIGHBORS = 1, 2, 4
STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EOVERFLOW", 5: "ESINGULAR", 6: "ETIMEOUT",
          7: "ENOACTIVESET", 8: "EUNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class MTPError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)}")


def header_functions():
    """Names of the functions declared in include/mtp.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\*?\s+\**(mtp_[a-z_0-9]+)\s*\(", text, re.M)))


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_L = ctypes.c_int64
_Z = ctypes.c_size_t

_SIGS = {
    "mtp_status_str": (ctypes.c_char_p, [_I]),
    "mtp_create": (_I, [_I, _I, _I, _D, _D, _P, _P, _I, ctypes.POINTER(_P)]),
    "mtp_destroy": (None, [_P]),
    "mtp_basis_count": (_I, [_P]),
    "mtp_radial_count": (_I, [_P]),
    "mtp_moment_count": (_I, [_P]),
    "mtp_level_table": (_I, [_P, _P, _Z, ctypes.POINTER(_Z)]),
    "mtp_set_params": (_I, [_P, _P, _P]),
    "mtp_set_neighbor_capacity": (_I, [_P, _I]),
    "mtp_last_neighbor_max": (_I, [_P]),
    "mtp_neighbors": (_I, [_P, _I, _I, _P, _P, _P, _D, _P, _P, _P, _P, _L, _I, _P]),
    "mtp_eval_batch": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _P]),
    "mtp_eval": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _P]),
    "mtp_sync": (_I, [_P, _P]),
    "mtp_launch_count": (_L, [_P]),
    "mtp_profile": (_I, [_P, _I]),
    "mtp_select_active_set": (_I, [_P, _I, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_D), _I, _P]),
    "mtp_set_active_set": (_I, [_P, _P]),
    "mtp_get_active_set": (_I, [_P, _P, _P, _P]),
    "mtp_grade": (_I, [_P, _I, _P, _P, _I, _P]),
    "mtp_param_grad": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _P, _P, _D, _D, _D, _I, _P, _P, _P, _I, _P]),
    "mtp_set_skin": (_I, [_P, _D]),
    "mtp_set_threads_per_atom": (_I, [_P, _I, _I]),
    "mtp_md_run": (_I, [_P, _I, _P, _P, _P, _P, _P, _D, _I, _P, _P, ctypes.POINTER(_I), _I, _P]),
    "mtp_select_active_set_noalloc": (_I, [_I, _I, _P, _P, _P, ctypes.POINTER(_I), _P]),
    "mtp_profile_read": (_I, [_P, _P, _I, ctypes.POINTER(_L)]),
    "mtp_save": (_I, [_P, ctypes.c_char_p]),
    "mtp_load": (_I, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    "mtp_fp32_peak": (_I, [_I, ctypes.POINTER(_D)]),
    "mtp_set_grade_kind": (_I, [_P, _I, _I, _P]),
    "mtp_train": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _P, _P, _D, _D, _D, _I, _I, _I, _D, _P,
                       ctypes.POINTER(_I), ctypes.POINTER(_I), _P]),
    "mtp_grade_columns": (_I, [_P, _P]),
    "mtp_relax_batch": (_I, [_P, _I, _I, _P, _P, _P, _P, _I, _D, _D, _D, _I, _D, _D, _P, _P, _P, _P]),
    "mtp_grade_width": (_I, [_P]),
    "mtp_jacobian_rows": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _I, _P]),
    "mtp_select_add": (_I, [_P, _I, _P, _P, ctypes.POINTER(_I), _P, ctypes.POINTER(_I), _I, _P]),
    "mtp_md_select": (_I, [_P, _I, _P, _P, _P, _P, _P, _D, _I, _D, _D, _I, _P, _P, _P, ctypes.POINTER(_I),
                           ctypes.POINTER(_I), _P, _P, _P, ctypes.POINTER(_I), _I, _P]),
    "mtp_autotune": (_I, [_P, _I, _I, _P, _P, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_I), _P, _P]),
}

PHASES = ("neighbors", "moments", "contract", "pairgrad", "gather")


def load():
    """Load the in-tree libmtp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmtp.so not built ({LIB_PATH}); run __graft_entry__.build()")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                if hasattr(lib, name):
                    fn = getattr(lib, name)
                    fn.restype = res
                    fn.argtypes = args
            _lib = lib
    return _lib


def _check(code, what):
    if code != 0:
        raise MTPError(code, what)


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def _stream(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# -- functions with the names of the C ABI (thin forwards) ---------------------------------------
def mtp_status_str(code):
    return load().mtp_status_str(code).decode()


def mtp_create(lev_max, n_species, n_radial, r_min, r_cut, xi=None, c=None, precision=FP64):
    lib = load()
    h = ctypes.c_void_p()
    xi_a = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64)
    c_a = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    _check(lib.mtp_create(int(lev_max), int(n_species), int(n_radial), float(r_min), float(r_cut), _ptr(xi_a),
                          _ptr(c_a), int(precision), ctypes.byref(h)), "mtp_create")
    return h


def mtp_destroy(h):
    load().mtp_destroy(h)


def mtp_level_table(h):
    lib = load()
    n = ctypes.c_size_t()
    _check(lib.mtp_level_table(h, None, 0, ctypes.byref(n)), "mtp_level_table")
    buf = np.zeros(n.value, dtype=np.int32)
    _check(lib.mtp_level_table(h, _ptr(buf), n.value, ctypes.byref(n)), "mtp_level_table")
    return buf


def mtp_set_params(h, xi=None, c=None):
    xi_a = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64)
    c_a = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    _check(load().mtp_set_params(h, _ptr(xi_a), _ptr(c_a)), "mtp_set_params")


def mtp_eval_batch(h, n_cfg, n_atoms, cfg_off, pos, types, cells, energy=None, forces=None, virial=None,
                   site_energy=None, b_rows=None, b_atoms=None, grade_cfg=None, grade_atom=None, flags=0,
                   stream=None):
    s = None if flags & HOST_MEMORY else _stream(stream)
    code = load().mtp_eval_batch(h, int(n_cfg), int(n_atoms), _ptr(cfg_off), _ptr(pos), _ptr(types), _ptr(cells),
                                 _ptr(energy), _ptr(forces), _ptr(virial), _ptr(site_energy), _ptr(b_rows),
                                 _ptr(b_atoms), _ptr(grade_cfg), _ptr(grade_atom), int(flags), s)
    _check(code, "mtp_eval_batch")


def mtp_neighbors(h, n_cfg, n_atoms, cfg_off, pos, cells, skin, counts, nbr_j=None, nbr_s=None, r_ij=None,
                  cap_pairs=0, flags=0, stream=None):
    code = load().mtp_neighbors(h, int(n_cfg), int(n_atoms), _ptr(cfg_off), _ptr(pos), _ptr(cells), float(skin),
                                _ptr(counts), _ptr(nbr_j), _ptr(nbr_s), _ptr(r_ij), int(cap_pairs), int(flags),
                                _stream(stream))
    _check(code, "mtp_neighbors")


def mtp_param_grad(h, n_cfg, n_atoms, cfg_off, pos, types, cells, e_ref, f_ref, w_ref, w_e, w_f, w_s, scaling,
                   loss=None, d_xi=None, d_c=None, flags=0, stream=None):
    s = None if flags & HOST_MEMORY else _stream(stream)
    _check(load().mtp_param_grad(h, int(n_cfg), int(n_atoms), _ptr(cfg_off), _ptr(pos), _ptr(types), _ptr(cells),
                                 _ptr(e_ref), _ptr(f_ref), _ptr(w_ref), float(w_e), float(w_f), float(w_s),
                                 int(scaling), _ptr(loss), _ptr(d_xi), _ptr(d_c), int(flags), s), "mtp_param_grad")


def mtp_set_skin(h, skin):
    _check(load().mtp_set_skin(h, float(skin)), "mtp_set_skin")


def mtp_set_threads_per_atom(h, moments, pairs):
    _check(load().mtp_set_threads_per_atom(h, int(moments), int(pairs)), "mtp_set_threads_per_atom")


def mtp_md_run(h, n_atoms, pos, vel, types, cell, masses, dt, n_steps, stream=None):
    """Velocity Verlet in place on device tensors; returns (e_pot [n+1], e_kin [n+1], rebuilds)."""
    ep = np.zeros(n_steps + 1)
    ek = np.zeros(n_steps + 1)
    nr = ctypes.c_int()
    m = np.ascontiguousarray(masses, dtype=np.float64)
    _check(load().mtp_md_run(h, int(n_atoms), _ptr(pos), _ptr(vel), _ptr(types), _ptr(cell), _ptr(m), float(dt),
                             int(n_steps), _ptr(ep), _ptr(ek), ctypes.byref(nr), 0, _stream(stream)), "mtp_md_run")
    return ep, ek, int(nr.value)


def mtp_select_add(h, m, n_cand, cand_rows, flags=0, stream=None):
    """Select-add update of the active set; returns (entered candidate indices, rows [m], swaps)."""
    entered = np.zeros(m, dtype=np.int32)
    rows = np.zeros(m, dtype=np.int32)
    ne, sw = ctypes.c_int(), ctypes.c_int()
    s = None if flags & HOST_MEMORY else _stream(stream)
    _check(load().mtp_select_add(h, int(n_cand), _ptr(cand_rows), _ptr(entered), ctypes.byref(ne), _ptr(rows),
                                 ctypes.byref(sw), int(flags), s), "mtp_select_add")
    return entered[:ne.value].tolist(), rows, int(sw.value)


def mtp_md_select(h, n_atoms, pos, vel, types, cell, masses, dt, n_steps, gamma_select, gamma_break, ring_pos,
                  stream=None):
    """MD with the two-threshold check (device tensors; ring_pos [cap, n, 3] float64 device).  Returns a
    dict: n_selected, stop_step (None if completed), ring_steps, ring_gamma, gammas, e_pot, e_kin, rebuilds."""
    cap = 0 if ring_pos is None else int(ring_pos.shape[0])
    rs = np.zeros(max(cap, 1), dtype=np.int32)
    rg = np.zeros(max(cap, 1))
    g = np.full(n_steps + 1, np.nan)
    ep = np.full(n_steps + 1, np.nan)
    ek = np.full(n_steps + 1, np.nan)
    ns, stop, nr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    m = np.ascontiguousarray(masses, dtype=np.float64)
    _check(load().mtp_md_select(h, int(n_atoms), _ptr(pos), _ptr(vel), _ptr(types), _ptr(cell), _ptr(m), float(dt),
                                int(n_steps), float(gamma_select), float(gamma_break), cap, _ptr(ring_pos),
                                _ptr(rs), _ptr(rg), ctypes.byref(ns), ctypes.byref(stop), _ptr(g), _ptr(ep), _ptr(ek),
                                ctypes.byref(nr), 0, _stream(stream)), "mtp_md_select")
    last = n_steps if stop.value < 0 else stop.value
    return {"n_selected": int(ns.value), "stop_step": None if stop.value < 0 else int(stop.value),
            "ring_steps": rs[:min(cap, ns.value)], "ring_gamma": rg[:min(cap, ns.value)], "gammas": g[:last + 1],
            "e_pot": ep[:last + 1], "e_kin": ek[:last + 1], "rebuilds": int(nr.value)}


def mtp_sync(h, stream=None):
    _check(load().mtp_sync(h, _stream(stream)), "mtp_sync")


def mtp_launch_count(h):
    return int(load().mtp_launch_count(h))


def mtp_select_active_set(h, n_rows, b_rows, selected=None, flags=0, stream=None):
    """Returns (number of swaps, final max |C|)."""
    sw = ctypes.c_int()
    g = ctypes.c_double()
    s = None if flags & HOST_MEMORY else _stream(stream)
    _check(load().mtp_select_active_set(h, int(n_rows), _ptr(b_rows), _ptr(selected), ctypes.byref(sw),
                                        ctypes.byref(g), int(flags), s), "mtp_select_active_set")
    return int(sw.value), float(g.value)


def mtp_select_active_set_noalloc(n_rows, m, b_rows, selected, a_inv=None, stream=None):
    """MaxVol with the library's fixed scratch array (no allocation); returns the number of swaps."""
    sw = ctypes.c_int()
    _check(load().mtp_select_active_set_noalloc(int(n_rows), int(m), _ptr(b_rows), _ptr(selected), _ptr(a_inv),
                                                ctypes.byref(sw), _stream(stream)), "mtp_select_active_set_noalloc")
    return int(sw.value)


def mtp_autotune(h, n_cfg, n_atoms, cfg_off, pos, types, cells, stream=None):
    """Times every lanes-per-atom choice on this batch; returns (moments, pairs, times_ms [4, 4])."""
    bm, bp = ctypes.c_int(), ctypes.c_int()
    t = np.zeros(16)
    _check(load().mtp_autotune(h, int(n_cfg), int(n_atoms), _ptr(cfg_off), _ptr(pos), _ptr(types), _ptr(cells),
                               ctypes.byref(bm), ctypes.byref(bp), _ptr(t), _stream(stream)), "mtp_autotune")
    return int(bm.value), int(bp.value), t.reshape(4, 4)


def mtp_fp32_peak(repeats=9):
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    t = ctypes.c_double()
    _check(load().mtp_fp32_peak(int(repeats), ctypes.byref(t)), "mtp_fp32_peak")
    return float(t.value)


def mtp_save(h, path):
    _check(load().mtp_save(h, os.fsencode(path)), "mtp_save")


def mtp_load(path):
    h = ctypes.c_void_p()
    _check(load().mtp_load(os.fsencode(path), ctypes.byref(h)), "mtp_load")
    return h


def mtp_set_active_set(h, A):
    _check(load().mtp_set_active_set(h, _ptr(np.ascontiguousarray(A, dtype=np.float64))), "mtp_set_active_set")


def mtp_get_active_set(h, m):
    A = np.zeros((m, m))
    Ai = np.zeros((m, m))
    rows = np.zeros(m, dtype=np.int32)
    _check(load().mtp_get_active_set(h, _ptr(A), _ptr(Ai), _ptr(rows)), "mtp_get_active_set")
    return A, Ai, rows


def mtp_grade(h, n_rows, b_rows, gamma, flags=0, stream=None):
    s = None if flags & HOST_MEMORY else _stream(stream)
    _check(load().mtp_grade(h, int(n_rows), _ptr(b_rows), _ptr(gamma), int(flags), s), "mtp_grade")


def mtp_profile(h, enable):
    _check(load().mtp_profile(h, int(bool(enable))), "mtp_profile")


def mtp_profile_read(h):
    """{phase: total ms} and the number of evaluations accumulated."""
    ms = np.zeros(len(PHASES))
    calls = ctypes.c_int64()
    _check(load().mtp_profile_read(h, _ptr(ms), len(PHASES), ctypes.byref(calls)), "mtp_profile_read")
    return dict(zip(PHASES, ms.tolist())), int(calls.value)


# -- convenience wrapper ----------------------------------------------------------------------------
class Model:
    """One potential on the current CUDA device (theta = {xi, c}, Sec. 2.1)."""

    def __init__(self, lev_max, n_species, n_radial, r_min, r_cut, xi=None, c=None, precision="fp64"):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.precision = prec
        self.n_species = int(n_species)
        self.n_radial = int(n_radial)
        self.h = mtp_create(lev_max, n_species, n_radial, r_min, r_cut, xi, c, prec)
        lib = load()
        self.m = lib.mtp_basis_count(self.h)
        self.n_mu = lib.mtp_radial_count(self.h)
        self.n_components = lib.mtp_moment_count(self.h)

    @classmethod
    def from_params(cls, p, precision="fp64"):
        return cls(p.lev_max, p.n_species, p.n_radial, p.r_min, p.r_cut, p.xi, p.c, precision)

    @classmethod
    def load(cls, path):
        """A model from a file written by save() (mtp_load)."""
        h = mtp_load(path)
        self = cls.__new__(cls)
        self.h = h
        lib = load()
        self.m = lib.mtp_basis_count(h)
        self.n_mu = lib.mtp_radial_count(h)
        self.n_components = lib.mtp_moment_count(h)
        # the file's header records the sizes that the handle does not expose
        head = {}
        with open(path) as f:
            for line in f:
                key, _, val = line.partition(" ")
                if key in ("n_species", "n_radial", "precision"):
                    head[key] = val.strip()
                if key == "xi":
                    break
        self.n_species = int(head["n_species"])
        self.n_radial = int(head["n_radial"])
        self.precision = PRECISIONS[head["precision"]]
        return self

    def save(self, path):
        mtp_save(self.h, path)

    def close(self):
        if getattr(self, "h", None):
            mtp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_table(self):
        return mtp_level_table(self.h)

    def set_params(self, xi=None, c=None):
        mtp_set_params(self.h, xi, c)

    def set_neighbor_capacity(self, cap):
        _check(load().mtp_set_neighbor_capacity(self.h, int(cap)), "mtp_set_neighbor_capacity")

    @property
    def launch_count(self):
        return mtp_launch_count(self.h)

    def eval_batch(self, pos, types, cells, cfg_off, forces=True, virial=True, site=False, b_rows=False,
                   b_atoms=False, grade_cfg=False, grade_atom=False, stream=None, flags=0, out=None):
        """Device tensors in (float64 pos [N,3], int32 types [N], float64 cells [K,3,3], int32 cfg_off [K+1]);
        device tensors out.  Passing back the dict of a previous call as `out` reuses its tensors, so that
        repeated calls have identical arguments (the library then replays its CUDA graph)."""
        import torch

        if out is not None:
            mtp_eval_batch(self.h, cells.shape[0], pos.shape[0], cfg_off, pos, types, cells, out["energy"],
                           out.get("forces"), out.get("virial"), out.get("site"), out.get("b_rows"), out.get("b_atoms"),
                           out.get("grade_cfg"), out.get("grade_atom"), flags, stream)
            return out
        dev = pos.device
        K = cells.shape[0]
        N = pos.shape[0]
        f64 = dict(dtype=torch.float64, device=dev)
        out = {"energy": torch.empty(K, **f64)}
        if forces:
            out["forces"] = torch.empty((N, 3), **f64)
        if virial:
            out["virial"] = torch.empty((K, 3, 3), **f64)
        if site:
            out["site"] = torch.empty(N, **f64)
        if b_rows:
            out["b_rows"] = torch.empty((K, self.m), **f64)
        if b_atoms:
            out["b_atoms"] = torch.empty((N, self.m), **f64)
        if grade_cfg:
            out["grade_cfg"] = torch.empty(K, **f64)
        if grade_atom:
            out["grade_atom"] = torch.empty(N, **f64)
        mtp_eval_batch(self.h, K, N, cfg_off, pos, types, cells, out["energy"], out.get("forces"), out.get("virial"),
                       out.get("site"), out.get("b_rows"), out.get("b_atoms"), out.get("grade_cfg"),
                       out.get("grade_atom"), flags, stream)
        return out

    def param_grad(self, pos, types, cells, cfg_off, e_ref, f_ref, w_ref, weights=(1.0, 0.01, 0.001),
                   scaling="vibrations"):
        """Loss and gradient (Sec. 2.2) for device tensors; returns (loss, d_xi [m], d_c [S,S,N_mu,N_Q])."""
        import torch

        kind = {"molecules": 0, "structures": 1, "vibrations": 2}[scaling] if isinstance(scaling, str) else scaling
        dev = pos.device
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        dxi = torch.empty(self.m, dtype=torch.float64, device=dev)
        S = self.n_species
        dc = torch.empty((S, S, self.n_mu, self.n_radial), dtype=torch.float64, device=dev)
        mtp_param_grad(self.h, cells.shape[0], pos.shape[0], cfg_off, pos, types, cells, e_ref, f_ref, w_ref,
                       weights[0], weights[1], weights[2], kind, loss, dxi, dc)
        return loss, dxi, dc

    def loss(self, pos, types, cells, cfg_off, e_ref, f_ref, w_ref, weights=(1.0, 0.01, 0.001),
             scaling="vibrations"):
        """The training loss alone (Sec. 2.2): the evaluation and the residuals, no gradient kernels."""
        import torch

        kind = {"molecules": 0, "structures": 1, "vibrations": 2}[scaling] if isinstance(scaling, str) else scaling
        loss = torch.empty(1, dtype=torch.float64, device=pos.device)
        mtp_param_grad(self.h, cells.shape[0], pos.shape[0], cfg_off, pos, types, cells, e_ref, f_ref, w_ref,
                       weights[0], weights[1], weights[2], kind, loss, None, None)
        return loss

    def set_skin(self, skin):
        mtp_set_skin(self.h, skin)

    def autotune(self, pos, types, cells, cfg_off):
        """Lanes per atom for batches of this size class (mtp_autotune); returns (moments, pairs, times_ms)."""
        return mtp_autotune(self.h, cells.shape[0], pos.shape[0], cfg_off, pos, types, cells)

    def set_threads_per_atom(self, moments=0, pairs=0):
        mtp_set_threads_per_atom(self.h, moments, pairs)

    def md_run(self, pos, vel, types, cell, masses, dt, n_steps, stream=None):
        """Velocity Verlet in place (device tensors); returns (e_pot, e_kin, rebuilds)."""
        return mtp_md_run(self.h, pos.shape[0], pos, vel, types, cell, masses, dt, n_steps, stream)

    def relax_batch(self, pos, types, cells, cfg_off, relax_cell=True, fmax=1e-4, smax=1e-5, gamma_break=float("inf"),
                    max_steps=5000, dt=0.05, dt_max=0.5):
        """FIRE relaxation of a batch in place (device tensors pos [N,3], cells [K,3,3]); returns
        (energy [K] device, steps [K], status [K]: 1 converged, 2 stopped by the grade, 3 step limit, 4 diverged)."""
        import torch

        K = cells.shape[0]
        energy = torch.empty(K, dtype=torch.float64, device=pos.device)
        steps = np.zeros(K, dtype=np.int32)
        status = np.zeros(K, dtype=np.int32)
        _check(load().mtp_relax_batch(self.h, K, pos.shape[0], _ptr(cfg_off), _ptr(pos), _ptr(types), _ptr(cells),
                                      int(bool(relax_cell)), float(fmax), float(smax), float(gamma_break),
                                      int(max_steps), float(dt), float(dt_max), _ptr(energy), _ptr(steps),
                                      _ptr(status), _stream(None)), "mtp_relax_batch")
        return energy, steps, status

    def train(self, pos, types, cells, cfg_off, e_ref, f_ref, w_ref, weights=(1.0, 0.01, 0.001),
              scaling="vibrations", history=10, max_iter=100, gtol=1e-8):
        """L-BFGS on the training loss (mtp_train); the model keeps the fitted parameters.
        Returns (losses per iterate, iterations, status: 0 converged, 1 max_iter, 2 line search)."""
        kind = {"molecules": 0, "structures": 1, "vibrations": 2}[scaling] if isinstance(scaling, str) else scaling
        losses = np.zeros(max_iter + 1)
        it, stt = ctypes.c_int(), ctypes.c_int()
        _check(load().mtp_train(self.h, cells.shape[0], pos.shape[0], _ptr(cfg_off), _ptr(pos), _ptr(types),
                                _ptr(cells), _ptr(e_ref), _ptr(f_ref), _ptr(w_ref), float(weights[0]),
                                float(weights[1]), float(weights[2]), int(kind), int(history), int(max_iter),
                                float(gtol), _ptr(losses), ctypes.byref(it), ctypes.byref(stt), _stream(None)),
               "mtp_train")
        return losses[:it.value + 1], int(it.value), int(stt.value)

    def set_grade_kind(self, nonlinear, cols=None):
        """0: grades of b rows (linear criterion); 1: grades of Jacobian rows dE/dtheta (nonlinear) over
        the parameter columns `cols` (ascending indices into [xi, c]; None = all)."""
        c = None if cols is None else np.ascontiguousarray(cols, dtype=np.int32)
        _check(load().mtp_set_grade_kind(self.h, int(nonlinear), 0 if c is None else len(c), _ptr(c)),
               "mtp_set_grade_kind")
        self.nonlinear = bool(nonlinear)

    @property
    def grade_width(self):
        return int(load().mtp_grade_width(self.h))

    def jacobian_rows(self, pos, types, cells, cfg_off):
        """Rows [K, m + S^2 N_mu N_Q] = [b(cfg), dE/dc] of the nonlinear criterion (device float64)."""
        import torch

        K = cells.shape[0]
        nonlin = getattr(self, "nonlinear", self.grade_width != self.m)
        w = self.grade_width if nonlin else self.m + self.n_species ** 2 * self.n_mu * self.n_radial
        rows = torch.empty((K, w), dtype=torch.float64, device=pos.device)
        _check(load().mtp_jacobian_rows(self.h, K, pos.shape[0], _ptr(cfg_off), _ptr(pos), _ptr(types), _ptr(cells),
                                        _ptr(rows), 0, _stream(None)), "mtp_jacobian_rows")
        return rows

    def select_add(self, cand_rows):
        """Select-add update from candidate b rows (device float64 [k, m]); (entered, rows, swaps)."""
        return mtp_select_add(self.h, self.grade_width, cand_rows.shape[0], cand_rows.contiguous())

    def md_select(self, pos, vel, types, cell, masses, dt, n_steps, gamma_select, gamma_break, ring_pos=None):
        return mtp_md_select(self.h, pos.shape[0], pos, vel, types, cell, masses, dt, n_steps, gamma_select,
                             gamma_break, ring_pos)

    def select_active_set(self, b_rows):
        """MaxVol over the rows of b_rows (device float64 [n, m]); returns (rows, swaps, max |C|)."""
        import torch

        sel = torch.empty(self.grade_width, dtype=torch.int32, device=b_rows.device)
        swaps, g = mtp_select_active_set(self.h, b_rows.shape[0], b_rows.contiguous(), sel)
        return sel, swaps, g

    def grade(self, b_rows):
        import torch

        g = torch.empty(b_rows.shape[0], dtype=torch.float64, device=b_rows.device)
        mtp_grade(self.h, b_rows.shape[0], b_rows.contiguous(), g)
        return g

    def eval(self, pos, types, cell, **kw):
        import torch

        off = torch.tensor([0, pos.shape[0]], dtype=torch.int32, device=pos.device)
        out = self.eval_batch(pos, types, cell.reshape(1, 3, 3), off, **kw)
        out["energy"] = out["energy"][0]
        if "virial" in out:
            out["virial"] = out["virial"][0]
        if "b_rows" in out:
            out["b_rows"] = out["b_rows"][0]
        return out

    def neighbors(self, pos, cells, cfg_off, skin=0.0):
        """Canonical neighbour lists: (counts [N], j [P], s [P,3], r_ij [P,3] float64), device tensors."""
        import torch

        N = pos.shape[0]
        K = cells.shape[0]
        counts = torch.empty(N, dtype=torch.int32, device=pos.device)
        mtp_neighbors(self.h, K, N, cfg_off, pos, cells, skin, counts)
        P = int(counts.sum().item())
        j = torch.empty(max(P, 1), dtype=torch.int32, device=pos.device)
        s = torch.empty((max(P, 1), 3), dtype=torch.int32, device=pos.device)
        r = torch.empty((max(P, 1), 3), dtype=torch.float64, device=pos.device)
        mtp_neighbors(self.h, K, N, cfg_off, pos, cells, skin, counts, j, s, r, P)
        return counts, j[:P], s[:P], r[:P]


# -- autograd ---------------------------------------------------------------------------------------
def _training_loss_function():
    import torch

    class TrainingLoss(torch.autograd.Function):
        """L(xi, c) of Sec. 2.2 (Eqs. 7, 11, 12) as a differentiable function of the parameters.

        forward: the library's evaluation and loss (mtp_param_grad without gradient outputs).
        backward: mtp_param_grad again, which re-evaluates energies, forces and virials (nothing of
        the forward pass is stored) and returns dL/dxi and dL/dc from the library's adjoint kernels,
        including the mixed second derivative of the force and stress terms.  xi [m] and c
        [S, S, N_mu, N_Q] are float64 tensors; they are copied into the model before each call."""

        @staticmethod
        def forward(ctx, xi, c, model, batch, refs, weights, scaling):
            model.set_params(xi.detach().double().cpu().numpy(), c.detach().double().cpu().numpy())
            loss = model.loss(*batch, *refs, weights=weights, scaling=scaling)
            ctx.save_for_backward(xi, c)
            ctx.model, ctx.batch, ctx.refs, ctx.weights, ctx.scaling = model, batch, refs, weights, scaling
            return loss[0].to(xi.device)

        @staticmethod
        def backward(ctx, grad_out):
            xi, c = ctx.saved_tensors
            model = ctx.model
            model.set_params(xi.detach().double().cpu().numpy(), c.detach().double().cpu().numpy())
            _, dxi, dc = model.param_grad(*ctx.batch, *ctx.refs, weights=ctx.weights, scaling=ctx.scaling)
            g = grad_out.to(dxi.device)
            return (g * dxi).to(xi.device), (g * dc).to(c.device), None, None, None, None, None

    return TrainingLoss


_TrainingLoss = None


def training_loss(model, xi, c, pos, types, cells, cfg_off, e_ref, f_ref, w_ref, weights=(1.0, 0.01, 0.001),
                  scaling="vibrations"):
    """Differentiable training loss: torch.autograd sees L(xi, c); backward runs the library's adjoint.
    Batch tensors as for Model.eval_batch, e_ref [K], f_ref [N, 3], w_ref [K, 9] (float64, device)."""
    global _TrainingLoss
    if _TrainingLoss is None:
        _TrainingLoss = _training_loss_function()
    return _TrainingLoss.apply(xi, c, model, (pos, types, cells, cfg_off), (e_ref, f_ref, w_ref), tuple(weights),
                               scaling)
