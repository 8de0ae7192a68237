"""The generated contraction parts of the float path, compiled for the host (g++, in double
precision: the part code is written for `float` and compiled here with float redefined as double).

For random moment values of a synthetic neighbourhood, for every partition into parts:
* the basis values B_alpha the parts write equal an independent full-Cartesian numpy.einsum
  contraction of the moment tensors for each graph of the oracle's level table (Sec. 2.1);
* the site-energy shares add up to V = sum_alpha xi_alpha B_alpha (Eq. 2);
* the dV/dM slots of each component add up to the derivative of V, checked by central differences.
No GPU.
"""

import ctypes
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
