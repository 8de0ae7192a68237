"""Host-side checks of the build-time generator (no GPU).

* the generator's level table equals the oracle's independent enumeration bit for bit;
* its contraction program, interpreted here with numpy on moments of a real neighbourhood,
  reproduces the oracle's basis values, and its adjoint program reproduces dV/dM (checked
  against the oracle's forces through the chain rule is done on the GPU; here against central
  differences of the interpreted forward program);
* the warp layouts cover every op exactly once, in dependency order.
"""

import numpy as np
import pytest

import oracle
from oracle import levels
from paper_2007_08555_gb300 import codegen, synth


@pytest.mark.parametrize("L", list(range(2, 22, 2)))
def test_level_table_bit_exact(L):
    assert codegen.level_table(codegen.build_basis(L)) == levels.level_table(L)


def _moments(prog, pot, p, cfg, atom):
    counts, j, s, d = oracle.neighbors(cfg.pos, cfg.cell, p.r_cut, which=[atom])
    zi = cfg.types[atom]
    mom = np.zeros(len(prog.comp_list))
    for jj, dd in zip(j, d):
        q, _ = pot.radial_basis(np.linalg.norm(dd))
        f = p.c[zi, cfg.types[jj]] @ q
        for k, (mu, (a, b, c)) in enumerate(prog.comp_list):
            mom[k] += f[mu] * dd[0] ** a * dd[1] ** b * dd[2] ** c
    return mom


def _forward(prog, mom):
    val = np.zeros(prog.n_values)
    val[:len(mom)] = mom
    for k, i, j, w in prog.ops:
        val[k] += w * val[i] * val[j]
    return val


@pytest.mark.parametrize("L", [8, 12, 16])
def test_program_reproduces_oracle_basis(L):
    prog = codegen.build_program(L)
    p = synth.random_params(L, 2, 6, 2.0, 5.0, prog.basis.m, seed=L)
    pot = oracle.Potential(p)
    cfg = synth.perturbed("fcc", (2, 2, 2), 0.15, np.random.default_rng(1), n_species=2)
    ref = pot.eval(cfg, want_b=True)["b_atoms"]
    for atom in (0, 9):
        val = _forward(prog, _moments(prog, pot, p, cfg, atom))
        got = val[prog.basis_value]
        np.testing.assert_allclose(got, ref[atom], rtol=1e-10, atol=1e-13 * np.abs(ref[atom]).max())


def _run_layout(rows, layers, val, seed, mode):
    """Interpret an encoded warp layout exactly as the kernel does."""
    out = seed.copy()
    for (start, end) in layers:
        acc = np.zeros(32)
        for r in range(start, end):
            for lane, (a, b, k, flags, w) in enumerate(rows[r]):
                if flags & 4:
                    continue
                if flags & 1:
                    acc[lane] = out[k] if mode == "adj" else 0.0
                if mode == "fwd":
                    acc[lane] += w * out[a] * out[b]
                else:
                    acc[lane] += w * val[a] * out[b]
                if flags & 2:
                    out[k] = acc[lane]
    return out


@pytest.mark.parametrize("L", [10, 16])
def test_warp_layouts_match_program(L):
    prog = codegen.build_program(L)
    rng = np.random.default_rng(3)
    mom = rng.normal(size=len(prog.comp_list))
    ref = _forward(prog, mom)
    rows, layers = codegen.encode_layout(codegen.forward_layout(prog))
    init = np.zeros(prog.n_values)
    init[:len(mom)] = mom
    got = _run_layout(rows, layers, None, init, "fwd")
    np.testing.assert_allclose(got, ref, rtol=1e-12)
    # adjoint: seed adj[basis value] = xi, then the reverse program gives dV/dval
    xi = rng.normal(size=prog.basis.m)
    seed = np.zeros(prog.n_values)
    for a, v in enumerate(prog.basis_value):
        seed[v] += xi[a]
    arows, alayers = codegen.encode_layout(codegen.adjoint_layout(prog))
    adj = _run_layout(arows, alayers, ref, seed, "adj")
    C = len(prog.comp_list)
    h = 1e-6
    for k in rng.choice(C, size=6, replace=False):
        mp = mom.copy()
        mp[k] += h
        mm = mom.copy()
        mm[k] -= h
        vp = _forward(prog, mp)[prog.basis_value] @ xi
        vm = _forward(prog, mm)[prog.basis_value] @ xi
        assert adj[k] == pytest.approx((vp - vm) / (2 * h), rel=1e-6, abs=1e-8)


def test_slices_partition_components():
    for L in (16, 20):
        prog = codegen.build_program(L)
        for cap in (codegen.SLICE_F32, codegen.SLICE_F64):
            sl = codegen.slices(prog, cap)
            flat = [i for _, comps in sl for i in comps]
            assert flat == list(range(len(prog.comp_list)))
            assert all(len(c) <= cap for _, c in sl)
