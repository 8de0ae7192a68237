"""The generated per-pair code compiled for the host (g++): for every slice, the adjoint (`grad`)
is the gradient of the moment accumulation (`mom`) contracted with dV/dM, and the tangent
functions of the loss gradient (`tmom`, `pdot`) are the directional derivatives they stand for.

For a pair r = (x, y, z) with radial values f_mu(|r|), `mom` accumulates the slice's moment
components M_t = f_mu(t) x^a y^b z^c (Eq. 5 for one neighbour); `grad` returns s and (gx, gy, gz)
such that d/dr sum_t adj_t M_t = (gx, gy, gz) + (s / |r|) r.  Checked by central differences in
double precision, for levels whose slices cover one or several groups of components.  No GPU.
"""

import ctypes
import shutil
import subprocess

import numpy as np
import pytest

from paper_2007_08555_gb300 import codegen

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


def _build(L, tmp_path):
    prog = codegen.build_program(L)
    slc = codegen.slices(prog, codegen.SLICE_F32)
    lines = codegen.emit_slice_functions(prog, slc, "f")
    n = len(slc)
    src = ["#define __device__", "#define __forceinline__ inline", "namespace gen {"] + lines + ["}"]
    sizes = ", ".join(f"gen::SliceF<{k}>::SIZE" for k in range(n))
    src.append(f'extern "C" int n_slices() {{ return {n}; }}')
    src.append(f'extern "C" int slice_size(int k) {{ static const int s[] = {{{sizes}}}; return s[k]; }}')
    src.append('extern "C" void mom(int k, double x, double y, double z, const double* f, double* acc) {')
    src.append("  switch (k) {")
    for k in range(n):
        src.append(f"    case {k}: gen::SliceF<{k}>::mom<double>(x, y, z, f, acc); break;")
    src.append("  }")
    src.append("}")
    src.append('extern "C" void grad(int k, double x, double y, double z, const double* f, const double* df, '
               "const double* adj, double* out) {")
    src.append("  double s = 0, gx = 0, gy = 0, gz = 0;")
    src.append("  switch (k) {")
    for k in range(n):
        src.append(f"    case {k}: gen::SliceF<{k}>::grad<double>(x, y, z, f, df, adj, s, gx, gy, gz); break;")
    src.append("  }")
    src.append("  out[0] = s; out[1] = gx; out[2] = gy; out[3] = gz;")
    src.append("}")
    src.append('extern "C" void tmom(int k, double x, double y, double z, const double* f, const double* df, '
               "double rdu, double ux, double uy, double uz, double* acc) {")
    src.append("  switch (k) {")
    for k in range(n):
        src.append(f"    case {k}: gen::SliceF<{k}>::tmom<double>(x, y, z, f, df, rdu, ux, uy, uz, acc); break;")
    src.append("  }")
    src.append("}")
    # pdot reads dV/dM and its tangent with the tile stride (32) from the slice's first component
    src.append('extern "C" void pdot(int k, double x, double y, double z, const double* adjp, const double* adjtp, '
               "double ux, double uy, double uz, double* P, double* Pd) {")
    src.append("  switch (k) {")
    for k in range(n):
        src.append(f"    case {k}: gen::SliceF<{k}>::pdot<double>(x, y, z, adjp, adjtp, ux, uy, uz, P, Pd); break;")
    src.append("  }")
    src.append("}")
    cpp = tmp_path / f"slices_L{L}.cpp"
    so = tmp_path / f"slices_L{L}.so"
    cpp.write_text("\n".join(src) + "\n")
    subprocess.run(["g++", "-O1", "-shared", "-fPIC", "-o", str(so), str(cpp)], check=True)
    lib = ctypes.CDLL(str(so))
    d = ctypes.c_double
    p = ctypes.POINTER(ctypes.c_double)
    lib.mom.argtypes = [ctypes.c_int, d, d, d, p, p]
    lib.grad.argtypes = [ctypes.c_int, d, d, d, p, p, p, p]
    lib.tmom.argtypes = [ctypes.c_int, d, d, d, p, p, d, d, d, d, p]
    lib.pdot.argtypes = [ctypes.c_int, d, d, d, p, p, d, d, d, p, p]
    return prog, lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@pytest.mark.parametrize("L", [10, 16, 20])
def test_grad_is_gradient_of_mom(L, tmp_path):
    prog, lib = _build(L, tmp_path)
    nmu = prog.n_mu
    rng = np.random.default_rng(L)
    a_mu = rng.uniform(0.5, 1.5, nmu)
    b_mu = rng.uniform(-1.0, 1.0, nmu)

    def radial(r):  # smooth stand-in radial functions and their derivatives
        return np.cos(a_mu * r + b_mu), -a_mu * np.sin(a_mu * r + b_mu)

    for k in range(lib.n_slices()):
        size = lib.slice_size(k)
        adj = rng.standard_normal(size)

        def value(v):
            f, _ = radial(float(np.linalg.norm(v)))
            f = np.ascontiguousarray(f)
            acc = np.zeros(size)
            lib.mom(k, v[0], v[1], v[2], _ptr(f), _ptr(acc))
            return float(adj @ acc)

        for _ in range(3):
            v = rng.standard_normal(3)
            v *= rng.uniform(1.5, 4.5) / np.linalg.norm(v)
            r = float(np.linalg.norm(v))
            f, df = (np.ascontiguousarray(t) for t in radial(r))
            out = np.zeros(4)
            lib.grad(k, v[0], v[1], v[2], _ptr(f), _ptr(df), _ptr(np.ascontiguousarray(adj)), _ptr(out))
            g = out[1:] + out[0] / r * v
            h = 1e-5 * r
            num = np.array([(value(v + h * e) - value(v - h * e)) / (2 * h) for e in np.eye(3)])
            scale = max(np.abs(num).max(), 1e-300)
            assert np.abs(g - num).max() <= 1e-6 * scale, (L, k, g, num)


def test_planted_sign_error_is_caught(tmp_path):
    """The check is sensitive: flipping the sign of the radial-derivative part fails it."""
    prog, lib = _build(10, tmp_path)
    nmu = prog.n_mu
    rng = np.random.default_rng(1)
    a_mu = rng.uniform(0.5, 1.5, nmu)
    size = lib.slice_size(0)
    adj = np.ascontiguousarray(rng.standard_normal(size))
    v = np.array([1.1, -0.7, 2.0])
    r = float(np.linalg.norm(v))
    f = np.ascontiguousarray(np.cos(a_mu * r))
    df = np.ascontiguousarray(-a_mu * np.sin(a_mu * r))
    out = np.zeros(4)
    lib.grad(0, v[0], v[1], v[2], _ptr(f), _ptr(df), _ptr(adj), _ptr(out))
    good = out[1:] + out[0] / r * v
    bad = out[1:] - out[0] / r * v

    def value(w):
        rr = float(np.linalg.norm(w))
        ff = np.ascontiguousarray(np.cos(a_mu * rr))
        acc = np.zeros(size)
        lib.mom(0, w[0], w[1], w[2], _ptr(ff), _ptr(acc))
        return float(adj @ acc)

    h = 1e-5
    num = np.array([(value(v + h * e) - value(v - h * e)) / (2 * h) for e in np.eye(3)])
    assert np.abs(good - num).max() <= 1e-6 * np.abs(num).max()
    assert np.abs(bad - num).max() > 1e-3 * np.abs(num).max()


@pytest.mark.parametrize("L", [10, 16, 20])
def test_tangent_moments_are_directional_derivatives(L, tmp_path):
    """tmom: the derivative of the slice's moment contributions along a pair displacement u."""
    prog, lib = _build(L, tmp_path)
    nmu = prog.n_mu
    rng = np.random.default_rng(100 + L)
    a_mu = rng.uniform(0.5, 1.5, nmu)

    def radial(r):
        return np.ascontiguousarray(np.cos(a_mu * r)), np.ascontiguousarray(-a_mu * np.sin(a_mu * r))

    for k in range(lib.n_slices()):
        size = lib.slice_size(k)

        def mom(v):
            acc = np.zeros(size)
            f, _ = radial(float(np.linalg.norm(v)))
            lib.mom(k, v[0], v[1], v[2], _ptr(f), _ptr(acc))
            return acc

        v = rng.standard_normal(3)
        v *= 3.0 / np.linalg.norm(v)
        u = rng.standard_normal(3)
        r = float(np.linalg.norm(v))
        f, df = radial(r)
        acc = np.zeros(size)
        lib.tmom(k, v[0], v[1], v[2], _ptr(f), _ptr(df), float(v @ u) / r, u[0], u[1], u[2], _ptr(acc))
        h = 1e-5
        num = (mom(v + h * u) - mom(v - h * u)) / (2 * h)
        assert np.abs(acc - num).max() <= 1e-6 * max(np.abs(num).max(), 1e-300), (L, k)


@pytest.mark.parametrize("L", [10, 16, 20])
def test_pdot_is_the_monomial_sum_and_its_tangent(L, tmp_path):
    """pdot: P_mu = sum_t adj_t mono_t over the components of radial index mu, and
    Pd_mu = sum_t adjt_t mono_t + d/de P_mu(r + e u)."""
    prog, lib = _build(L, tmp_path)
    nmu = prog.n_mu
    rng = np.random.default_rng(200 + L)
    for k in range(lib.n_slices()):
        size = lib.slice_size(k)

        def P_of(v, adj):
            # mom with f = e_mu picks out the components of radial index mu: P_mu = adj . acc
            out = np.zeros(nmu)
            for mu in range(nmu):
                e = np.zeros(nmu)
                e[mu] = 1.0
                acc = np.zeros(size)
                lib.mom(k, v[0], v[1], v[2], _ptr(e), _ptr(acc))
                out[mu] = adj @ acc
            return out

        adj = rng.standard_normal(size)
        adjt = rng.standard_normal(size)
        tile = np.zeros(size * 32)
        tile_t = np.zeros(size * 32)
        tile[::32] = adj
        tile_t[::32] = adjt
        v = rng.standard_normal(3) * 1.7
        u = rng.standard_normal(3)
        P = np.zeros(nmu)
        Pd = np.zeros(nmu)
        lib.pdot(k, v[0], v[1], v[2], _ptr(tile), _ptr(tile_t), u[0], u[1], u[2], _ptr(P), _ptr(Pd))
        np.testing.assert_allclose(P, P_of(v, adj), rtol=1e-12, atol=1e-12 * np.abs(P).max())
        h = 1e-5
        num = P_of(v, adjt) + (P_of(v + h * u, adj) - P_of(v - h * u, adj)) / (2 * h)
        assert np.abs(Pd - num).max() <= 1e-6 * max(np.abs(num).max(), 1e-300), (L, k)


@pytest.mark.parametrize("L", [16, 18, 20])
def test_moment_slices_accumulate_the_same_components(L, tmp_path):
    """The float moments kernel has its own slicing (as many slices, sizes balanced); concatenated,
    its slices accumulate exactly the components of the other kernels' slices, in storage order."""
    prog = codegen.build_program(L)
    s32 = codegen.slices(prog, codegen.SLICE_F32)
    sm32 = codegen.moment_slices(prog, codegen.SLICE_F32)
    assert len(sm32) == len(s32)
    assert [i for _, c in sm32 for i in c] == list(range(len(prog.comp_list)))
    assert max(len(c) for _, c in sm32) <= max(len(c) for _, c in s32)
    lines = codegen.emit_slice_functions(prog, s32, "f") + codegen.emit_slice_functions(prog, sm32, "mf")
    src = ["#define __device__", "#define __forceinline__ inline", "namespace gen {"] + lines + ["}"]
    for name, slc in (("f", s32), ("mf", sm32)):
        tag = "SliceF" if name == "f" else "SliceMF"
        src.append(f'extern "C" void all_{name}(double x, double y, double z, const double* f, double* acc) {{')
        for k, (_, comps) in enumerate(slc):
            src.append(f"  gen::{tag}<{k}>::mom<double>(x, y, z, f, acc + {min(comps)});")
        src.append("}")
    cpp = tmp_path / f"mslices_L{L}.cpp"
    so = tmp_path / f"mslices_L{L}.so"
    cpp.write_text("\n".join(src) + "\n")
    subprocess.run(["g++", "-O1", "-shared", "-fPIC", "-o", str(so), str(cpp)], check=True)
    lib = ctypes.CDLL(str(so))
    d = ctypes.c_double
    p = ctypes.POINTER(ctypes.c_double)
    lib.all_f.argtypes = lib.all_mf.argtypes = [d, d, d, p, p]
    rng = np.random.default_rng(L)
    C = len(prog.comp_list)
    for _ in range(4):
        v = rng.standard_normal(3) * 1.9
        f = np.ascontiguousarray(rng.standard_normal(prog.n_mu))
        a = np.zeros(C)
        b = np.zeros(C)
        lib.all_f(v[0], v[1], v[2], _ptr(f), _ptr(a))
        lib.all_mf(v[0], v[1], v[2], _ptr(f), _ptr(b))
        assert np.array_equal(a, b)
        # and each component is f_mu x^a y^b z^c
        ref = np.array([f[mu] * v[0] ** m[0] * v[1] ** m[1] * v[2] ** m[2] for mu, m in prog.comp_list])
        np.testing.assert_allclose(b, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
