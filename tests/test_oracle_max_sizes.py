"""Oracle pins at the largest sizes the library accepts: 8 species and N_Q = 16 radial functions
(Sec. 2.1, Eqs. 3-5).  The same checks as at small sizes, so that a later GPU parity case at these
sizes compares against a pinned reference: the Chebyshev identity up to T_15, the isolated-pair
closed form for the last species pairs, a full-Cartesian einsum of every basis function, species
relabelling with equal radial blocks, and forces as central differences of the energy."""

import numpy as np
import pytest

import oracle
from oracle import levels
from paper_2007_08555_gb300 import synth
from test_oracle_eval import _einsum_basis, _f_mu

S_MAX, NQ_MAX = 8, 16


def _params(L, seed):
    return synth.random_params(L, S_MAX, NQ_MAX, 2.0, 5.0, len(levels.basis(L)), seed)


def _cfg(seed, sigma=0.12):
    return synth.perturbed("fcc", (2, 2, 2), sigma, np.random.default_rng(seed), n_species=S_MAX)


def test_chebyshev_identity_up_to_t15():
    pot = oracle.Potential(_params(10, 1))
    for r in np.linspace(2.0, 4.99, 23):
        x = (2 * r - 7.0) / 3.0
        q, _ = pot.radial_basis(r)
        expect = np.cos(np.arange(NQ_MAX) * np.arccos(x)) * (5.0 - r) ** 2
        np.testing.assert_allclose(q, expect, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("zi,zj", [(7, 6), (0, 7)])
def test_isolated_pair_closed_form_last_species(zi, zj):
    L = 10
    p = _params(L, 2)
    pot = oracle.Potential(p)
    d = np.array([1.4, -2.2, 1.6])
    cfg = synth.Config(np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0]]) + np.array([[0, 0, 0], d]),
                       np.array([zi, zj], dtype=np.int32), np.eye(3) * 40.0)
    out = pot.eval(cfg, want_b=True)
    r = np.linalg.norm(d)
    comps = levels.connected_components(L)
    for i, (a, b) in enumerate([(zi, zj), (zj, zi)]):
        f = _f_mu(pot, p.c, a, b, r)
        expect = []
        for bf in levels.basis(L):
            v = 1.0
            for k in bf.components:
                for mu, nu in comps[k].labels:
                    v *= f[mu] * r**nu
            expect.append(v)
        np.testing.assert_allclose(out["b_atoms"][i], expect, rtol=1e-10)


def test_contractions_equal_full_cartesian_einsum():
    L = 10
    p = _params(L, 3)
    pot = oracle.Potential(p)
    cfg = _cfg(4)
    assert len(set(cfg.types.tolist())) >= 5
    out = pot.eval(cfg, want_b=True)
    for atom in (0, 17):
        ref = _einsum_basis(pot, p, cfg, atom, L)
        np.testing.assert_allclose(out["b_atoms"][atom], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_species_relabelling_with_equal_radial_blocks():
    p = _params(10, 5)
    p.c[:] = p.c[0, 0]
    pot = oracle.Potential(p)
    cfg = _cfg(6)
    relabel = np.random.default_rng(7).permutation(S_MAX).astype(np.int32)
    a = pot.eval(cfg)["energy"]
    b = pot.eval(synth.Config(cfg.pos, relabel[cfg.types], cfg.cell))["energy"]
    assert a == pytest.approx(b, rel=1e-12)


def test_forces_are_finite_differences():
    p = _params(10, 8)
    pot = oracle.Potential(p)
    cfg = _cfg(9)
    F = pot.eval(cfg)["forces"]
    rms = np.sqrt(np.mean(F**2))
    assert np.abs(F.sum(0)).max() <= 1e-11 * cfg.n * rms
    h = 1e-5
    for i, k in [(0, 0), (9, 1), (30, 2)]:
        pp, pm = cfg.pos.copy(), cfg.pos.copy()
        pp[i, k] += h
        pm[i, k] -= h
        fd = -(pot.eval(synth.Config(pp, cfg.types, cfg.cell))["energy"]
               - pot.eval(synth.Config(pm, cfg.types, cfg.cell))["energy"]) / (2 * h)
        assert abs(fd - F[i, k]) <= 1e-6 * rms
