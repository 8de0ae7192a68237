"""The generated contraction parts of the float path, compiled for the host (g++, in double
precision: the part code is written for `float` and compiled here with float redefined as double).

For random moment values of a synthetic neighbourhood, for every partition into parts:
* the basis values B_alpha the parts write equal an independent full-Cartesian numpy.einsum
  contraction of the moment tensors for each graph of the oracle's level table (Sec. 2.1);
* the site-energy shares add up to V = sum_alpha xi_alpha B_alpha (Eq. 2);
* the dV/dM slots of each component add up to the derivative of V, checked by central differences;
and for the tangent parts of the loss gradient, the per-basis terms ek B - dB/de along a moment
tangent T and the tangent dV/dM slots, against central differences.  No GPU.
"""

import ctypes
import itertools
import shutil
import string
import subprocess

import numpy as np
import pytest

from oracle import levels
from paper_2007_08555_gb300 import codegen

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


def _build(L, parts, tmp_path):
    prog = codegen.build_program(L)
    lines = codegen.emit_parts(prog, parts)
    C = len(prog.comp_list)
    src = ["#include <cstddef>", "#define __device__", "#define __forceinline__ inline", "#define float double",
           "namespace gen {"] + lines + ["}"]
    src.append('extern "C" double run_part(int g, const double* s, double* d, const double* xi, double* b) {')
    src.append("  return gen::contract_part<true>(g, s, d, xi, b);")
    src.append("}")
    src.append(f'extern "C" int slot_begin_at(int c) {{ return c <= {C} ? gen::slot_begin[c] : -1; }}')
    src.append('extern "C" int n_slots() { return gen::NSLOT; }')
    cpp = tmp_path / f"parts_L{L}_{parts}.cpp"
    so = tmp_path / f"parts_L{L}_{parts}.so"
    cpp.write_text("\n".join(src) + "\n")
    subprocess.run(["g++", "-O1", "-shared", "-fPIC", "-o", str(so), str(cpp)], check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.POINTER(ctypes.c_double)
    lib.run_part.restype = ctypes.c_double
    lib.run_part.argtypes = [ctypes.c_int, p, p, p, p]
    return prog, lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _neighbourhood(L, rng, n_pairs=7):
    """Cartesian moment tensors M[(mu, nu)] = sum_j f_mu(j) d_j^{(x) nu} of random pairs."""
    numax = max(nu for _, nu in levels.used_moments(L))
    nmu = max(mu for mu, _ in levels.used_moments(L)) + 1
    d = rng.normal(size=(n_pairs, 3)) * 0.7
    f = rng.normal(size=(n_pairs, nmu)) * 0.8
    M = {}
    for mu in range(nmu):
        for nu in range(numax + 1):
            t = np.zeros((3,) * nu)
            for j in range(n_pairs):
                o = np.array(1.0)
                for _ in range(nu):
                    o = np.multiply.outer(o, d[j])
                t = t + f[j, mu] * o
            M[(mu, nu)] = t
    return M


def _einsum_basis(M, L):
    comps = levels.connected_components(L)
    vals = []
    for c in comps:
        a = c.matrix()
        letters = iter(string.ascii_letters)
        subs = [[] for _ in range(c.n)]
        for u in range(c.n):
            for v in range(u + 1, c.n):
                for _ in range(a[u][v]):
                    ch = next(letters)
                    subs[u].append(ch)
                    subs[v].append(ch)
        expr = ",".join("".join(s) for s in subs) + "->"
        vals.append(float(np.einsum(expr, *[M[lab] for lab in c.labels])))
    return np.array([np.prod([vals[k] for k in b.components]) for b in levels.basis(L)])


def _tile(prog, M):
    """Moment components in the tile layout of one atom (component c at [c * 32])."""
    src = np.zeros(len(prog.comp_list) * 32)
    for c, (mu, (a, b, cc)) in enumerate(prog.comp_list):
        idx = (0,) * a + (1,) * b + (2,) * cc
        src[c * 32] = M[(mu, a + b + cc)][idx] if idx else M[(mu, 0)]
    return src


def _run(lib, prog, parts, src, xi):
    m = len(xi)
    dst = np.zeros(lib.n_slots() * 32)
    b = np.full(m, np.nan)
    e = sum(lib.run_part(g, _ptr(src), _ptr(dst), _ptr(xi), _ptr(b)) for g in range(parts))
    C = len(prog.comp_list)
    adj = np.array([dst[[s * 32 for s in range(lib.slot_begin_at(c), lib.slot_begin_at(c + 1))]].sum()
                    for c in range(C)])
    return e, b, adj


@pytest.mark.parametrize("L,parts", [(10, 1), (12, 2), (16, 1), (16, 4), (16, 8), (20, 8)])
def test_parts_evaluate_the_basis_and_its_adjoint(L, parts, tmp_path):
    prog, lib = _build(L, parts, tmp_path)
    rng = np.random.default_rng(L * 10 + parts)
    M = _neighbourhood(L, rng)
    src = _tile(prog, M)
    m = len(levels.basis(L))
    xi = rng.normal(size=m)
    e, b, adj = _run(lib, prog, parts, src, xi)
    ref = _einsum_basis(M, L)
    assert not np.isnan(b).any(), "every basis function is written by exactly one part"
    np.testing.assert_allclose(b, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    assert e == pytest.approx(float(xi @ ref), rel=1e-10)
    # dV/dM of every component against central differences of the site energy
    scale = np.abs(src).max()
    for c in range(len(prog.comp_list)):
        h = 1e-6 * max(abs(src[c * 32]), scale)
        sp, sm = src.copy(), src.copy()
        sp[c * 32] += h
        sm[c * 32] -= h
        ep = _run(lib, prog, parts, sp, xi)[0]
        em = _run(lib, prog, parts, sm, xi)[0]
        num = (ep - em) / (2 * h)
        assert adj[c] == pytest.approx(num, rel=1e-6, abs=1e-7 * max(abs(e) / scale, 1e-12)), (L, parts, c)


def _build_dual(L, parts, tmp_path):
    prog = codegen.build_program(L)
    lines = codegen.emit_dual_parts(prog, parts)
    C = len(prog.comp_list)
    # one lane: the warp sum of a lane's term is the term itself (the other lanes add zeros)
    src = ["#include <cstddef>", "#define __device__", "#define __forceinline__ inline", "#define float double",
           "inline double __shfl_xor_sync(unsigned, double, int) { return 0.0; }", "namespace gen {"] + lines + ["}"]
    src.append('extern "C" void run_dual(int g, const double* m, const double* mt, double* adj, double* adt, '
               "const double* xi, double ek, double* dxt) {")
    src.append("  gen::dual_part(g, m, mt, adj, adt, xi, ek, true, true, dxt);")
    src.append("}")
    src.append(f'extern "C" int dslot_begin_at(int c) {{ return c <= {C} ? gen::dslot_begin[c] : -1; }}')
    src.append('extern "C" int n_dslots() { return gen::NDSLOT; }')
    cpp = tmp_path / f"dual_L{L}_{parts}.cpp"
    so = tmp_path / f"dual_L{L}_{parts}.so"
    cpp.write_text("\n".join(src) + "\n")
    subprocess.run(["g++", "-O1", "-shared", "-fPIC", "-o", str(so), str(cpp)], check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.POINTER(ctypes.c_double)
    lib.run_dual.restype = None
    lib.run_dual.argtypes = [ctypes.c_int, p, p, p, p, p, ctypes.c_double, p]
    return prog, lib


def _run_dual(lib, prog, parts, m_tile, t_tile, xi, ek):
    nd = lib.n_dslots()
    adj, adt = np.zeros(nd * 32), np.zeros(nd * 32)
    dxt = np.full(len(xi), np.nan)
    for g in range(parts):
        lib.run_dual(g, _ptr(m_tile), _ptr(t_tile), _ptr(adj), _ptr(adt), _ptr(xi), ek, _ptr(dxt))
    C = len(prog.comp_list)

    def per_comp(a):
        return np.array([a[[s * 32 for s in range(lib.dslot_begin_at(c), lib.dslot_begin_at(c + 1))]].sum()
                         for c in range(C)])

    return per_comp(adj), per_comp(adt), dxt


@pytest.mark.parametrize("L,parts", [(10, 1), (12, 2), (16, 8)])
def test_dual_parts_are_the_tangent_contraction(L, parts, tmp_path):
    """dxt_alpha = ek B_alpha - dB_alpha/de (M + e T); the dV/dM slots add up to dV/dM and the tangent
    slots to its directional derivative along T (central differences of the value and adjoint)."""
    prog, lib = _build_dual(L, parts, tmp_path)
    rng = np.random.default_rng(L * 100 + parts)
    M = _neighbourhood(L, rng)
    m_tile = _tile(prog, M)
    C = len(prog.comp_list)
    t_tile = np.zeros_like(m_tile)
    t_tile[::32] = rng.normal(size=C) * np.abs(m_tile[::32]).mean()
    m = len(levels.basis(L))
    xi = rng.normal(size=m)
    ek = 0.37
    adj, adt, dxt = _run_dual(lib, prog, parts, m_tile, t_tile, xi, ek)
    assert not np.isnan(dxt).any(), "every basis function is written by exactly one part"

    def comps_to_cart(tile):
        # moment tensors from tile values: the symmetric tensor with the given components
        out = {}
        for c, (mu, (a, b, cc)) in enumerate(prog.comp_list):
            nu = a + b + cc
            key = (mu, nu)
            if key not in out:
                out[key] = np.zeros((3,) * nu)
            for idx in set(itertools.permutations((0,) * a + (1,) * b + (2,) * cc)):
                out[key][idx] = tile[c * 32]
        for key, val in M.items():
            out.setdefault(key, val)
        return out

    h = 1e-6
    Bp = _einsum_basis(comps_to_cart(m_tile + h * t_tile), L)
    Bm = _einsum_basis(comps_to_cart(m_tile - h * t_tile), L)
    B0 = _einsum_basis(comps_to_cart(m_tile), L)
    np.testing.assert_allclose(B0, _einsum_basis(M, L), rtol=1e-12, atol=1e-14 * np.abs(B0).max())
    ref = ek * B0 - (Bp - Bm) / (2 * h)
    np.testing.assert_allclose(dxt, ref, rtol=1e-6, atol=1e-7 * np.abs(ref).max())
    # tangent slots: the directional derivative of the dV/dM slots computed by the same code
    ap = _run_dual(lib, prog, parts, m_tile + h * t_tile, t_tile, xi, ek)[0]
    am = _run_dual(lib, prog, parts, m_tile - h * t_tile, t_tile, xi, ek)[0]
    np.testing.assert_allclose(adt, (ap - am) / (2 * h), rtol=1e-6, atol=1e-7 * np.abs(adt).max())
    # and the dV/dM slots equal those of the forward parts (which are pinned above)
    _, fl = _build(L, codegen.CONTRACT_PARTS[L], tmp_path)
    _, _, adj_f = _run(fl, prog, codegen.CONTRACT_PARTS[L], m_tile, xi)
    np.testing.assert_allclose(adj, adj_f, rtol=1e-12, atol=1e-12 * np.abs(adj_f).max())


@pytest.mark.parametrize("L,lanes", [(18, 2), (20, 2), (20, 8), (16, 4)])
def test_adjoint_slots_into_shared_arrays(L, lanes, tmp_path):
    """The pair-gradient kernel gathers dV/dM of an atom from the contraction parts' slots into shared
    memory: per slice (OFF = 0, positions 0 .. SIZE-1) or, for all slices at once, at the components'
    own positions (OFF = BEGIN).  Both give every component the sum of its slots, in vectors of four
    components NS atoms apart, each written by exactly one of the atom's lanes."""
    prog = codegen.build_program(L)
    parts = codegen.CONTRACT_PARTS[L]
    part_lines = codegen.emit_parts(prog, parts)
    slot_begin = [int(x) for x in part_lines[2].split("{")[1].rstrip("};").split(",")]
    slc = codegen.slices(prog, codegen.SLICE_F32)
    lines = codegen.emit_slice_functions(prog, slc, "f", slot_begin)
    NS = 128 // lanes
    C = len(prog.comp_list)
    src = ["#define __device__", "#define __forceinline__ inline", "namespace gen {"] + lines + ["}"]
    src.append('extern "C" void gather(int merged, int k, int sub, const double* sl, double* dst) {')
    src.append("  switch (k) {")
    for k, (_, comps) in enumerate(slc):
        off = f"gen::SliceF<{k}>::BEGIN"
        src.append(f"    case {k}: if (merged) gen::SliceF<{k}>::adj_to_shared<double, {lanes}, {NS}, {off}>(sl, dst, sub);"
                   f" else gen::SliceF<{k}>::adj_to_shared<double, {lanes}, {NS}>(sl, dst, sub); break;")
    src.append("  }")
    src.append("}")
    cpp = tmp_path / f"adjsh_L{L}.cpp"
    so = tmp_path / f"adjsh_L{L}.so"
    cpp.write_text("\n".join(src) + "\n")
    subprocess.run(["g++", "-O1", "-shared", "-fPIC", "-o", str(so), str(cpp)], check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.POINTER(ctypes.c_double)
    lib.gather.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, p, p]
    rng = np.random.default_rng(L + lanes)
    nslot = slot_begin[-1]
    sl = np.zeros(nslot * 32)
    sl[::32] = rng.standard_normal(nslot)  # this atom's slots (tile stride 32)
    want = np.array([sl[[s * 32 for s in range(slot_begin[c], slot_begin[c + 1])]].sum() for c in range(C)])

    def at(pos):  # element of component position pos in the atom's strided vectors
        return (pos // 4) * 4 * NS + pos % 4

    size = ((C + 3) // 4) * 4 * NS
    merged = np.full(size, np.nan)
    for k, (_, comps) in enumerate(slc):
        per = np.full(((len(comps) + 3) // 4) * 4 * NS, np.nan)
        for sub in range(lanes):
            lib.gather(0, k, sub, sl.ctypes.data_as(p), per.ctypes.data_as(p))
            lib.gather(1, k, sub, sl.ctypes.data_as(p), merged.ctypes.data_as(p))
        got = np.array([per[at(t)] for t in range(len(comps))])
        np.testing.assert_allclose(got, want[comps], rtol=1e-13, atol=0)
    np.testing.assert_allclose(np.array([merged[at(c)] for c in range(C)]), want, rtol=1e-13, atol=0)
    # nothing written outside the components' positions (other atoms' vectors stay untouched)
    touched = {at(c) for c in range(C)}
    assert all(np.isnan(merged[i]) for i in range(size) if i not in touched)
    # each position by exactly one lane of the atom
    written = []
    for sub in range(lanes):
        one = np.full(size, np.nan)
        for k in range(len(slc)):
            lib.gather(1, k, sub, sl.ctypes.data_as(p), one.ctypes.data_as(p))
        written.append(set(np.flatnonzero(~np.isnan(one)).tolist()))
    assert sum(len(w) for w in written) == C and set().union(*written) == touched
