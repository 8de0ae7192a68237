"""Pins of the oracle's energy, forces and virial (Sec. 2.1, Eqs. 1-4), against what the
mathematics fixes rather than against the oracle itself:

* Chebyshev radial basis: T_n(cos t) = cos(n t), the (R_cut - r)^2 factor, dQ/dr by finite differences;
* isolated pair: every basis function equals prod_k f_{mu_k}(r) * r^(sum nu) (one neighbour makes
  every contracted index pair an r.r);
* every basis function equals an independent full-Cartesian numpy.einsum contraction of the
  3^nu moment tensors (lev_max 10 and 12);
* invariance of E under rotations, reflections, translations and same-species permutations
  (Sec. 2.1); the virial rotates as R W R^T;
* forces equal central finite differences of E and sum to zero; the virial equals the finite
  difference of E under a homogeneous strain and is symmetric;
* E and F go to zero as a pair separates to R_cut, as delta^2 and delta (Eq. 4);
* extensivity of E and W over supercells of small cells (periodic images);
* neighbour lists equal an independent numpy brute force over a wide image range.
"""

import itertools
import string

import numpy as np
import pytest

import oracle
from oracle import levels
from paper_2007_08555_gb300 import synth


def _params(L, S=1, seed=0, NQ=8, xi_std=1e-2, c_std=0.1):
    return synth.random_params(L, S, NQ, 2.0, 5.0, len(levels.basis(L)), seed, xi_std, c_std)


def _small_cfg(seed=7, kind="fcc", reps=(2, 2, 2), sigma=0.12, S=1):
    rng = np.random.default_rng(seed)
    return synth.perturbed(kind, reps, sigma, rng, n_species=S)


def test_radial_basis_chebyshev_identity_and_derivative():
    pot = oracle.Potential(_params(10))
    rmin, rcut = 2.0, 5.0
    for r in np.linspace(1.2, 4.99, 37):
        x = (2 * r - rmin - rcut) / (rcut - rmin)
        q, dq = pot.radial_basis(r)
        if abs(x) <= 1:
            t = np.arccos(x)
            expect = np.cos(np.arange(8) * t) * (rcut - r) ** 2
            np.testing.assert_allclose(q, expect, rtol=1e-12, atol=1e-12)
        h = 1e-6
        qp, _ = pot.radial_basis(r + h)
        qm, _ = pot.radial_basis(r - h)
        np.testing.assert_allclose(dq, (qp - qm) / (2 * h), rtol=1e-6, atol=1e-6)
    q, _ = pot.radial_basis(rcut)
    assert np.all(q == 0.0)


def _f_mu(pot, c, zi, zj, r):
    q, _ = pot.radial_basis(r)
    return c[zi, zj] @ q


@pytest.mark.parametrize("L", [8, 12, 16])
def test_isolated_pair_closed_form(L):
    p = _params(L, S=2, seed=3)
    pot = oracle.Potential(p)
    cell = np.eye(3) * 40.0
    d = np.array([1.7, -2.1, 1.3])
    cfg = synth.Config(np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0]]) + np.array([[0, 0, 0], d]),
                       np.array([0, 1], dtype=np.int32), cell)
    out = pot.eval(cfg, want_b=True)
    r = np.linalg.norm(d)
    comps = levels.connected_components(L)
    for i, (zi, zj) in enumerate([(0, 1), (1, 0)]):
        f = _f_mu(pot, p.c, zi, zj, r)
        expect = []
        for b in levels.basis(L):
            v = 1.0
            for k in b.components:
                for mu, nu in comps[k].labels:
                    v *= f[mu] * r**nu
            expect.append(v)
        np.testing.assert_allclose(out["b_atoms"][i], expect, rtol=1e-11)
        assert out["site"][i] == pytest.approx(float(np.dot(p.xi, expect)), rel=1e-11)


def _einsum_basis(pot, p, cfg, atom, L):
    """Full-Cartesian basis values of one neighbourhood, written independently with numpy."""
    counts, j, s, d = oracle.neighbors(cfg.pos, cfg.cell, p.r_cut, which=[atom])
    zi = cfg.types[atom]
    numax = max(nu for _, nu in levels.used_moments(L))
    nmu = synth.n_mu(L)
    M = {}
    for mu in range(nmu):
        for nu in range(numax + 1):
            M[(mu, nu)] = np.zeros((3,) * nu)
    for jj, dd in zip(j, d):
        f = _f_mu(pot, p.c, zi, cfg.types[jj], np.linalg.norm(dd))
        t = np.array(1.0)
        outer = [t]
        for nu in range(1, numax + 1):
            t = np.multiply.outer(t, dd)
            outer.append(t)
        for mu in range(nmu):
            for nu in range(numax + 1):
                M[(mu, nu)] = M[(mu, nu)] + f[mu] * outer[nu]
    comps = levels.connected_components(L)
    cvals = []
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
        expr = ",".join("".join(sub) for sub in subs) + "->"
        cvals.append(float(np.einsum(expr, *[M[lab] for lab in c.labels])))
    return np.array([np.prod([cvals[k] for k in b.components]) for b in levels.basis(L)])


@pytest.mark.parametrize("L", [10, 12])
def test_contractions_equal_full_cartesian_einsum(L):
    p = _params(L, S=2, seed=5)
    pot = oracle.Potential(p)
    cfg = _small_cfg(seed=11, S=2)
    out = pot.eval(cfg, want_b=True)
    for atom in (0, 13):
        ref = _einsum_basis(pot, p, cfg, atom, L)
        np.testing.assert_allclose(out["b_atoms"][atom], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.fixture(scope="module")
def pot12():
    p = _params(12, S=2, seed=9)
    return p, oracle.Potential(p)


def test_rotation_reflection_translation_invariance(pot12):
    p, pot = pot12
    cfg = _small_cfg(seed=21, S=2)
    base = pot.eval(cfg)
    for seed, refl in [(1, False), (2, True)]:
        R = synth.rotation(seed, reflect=refl)
        rc = synth.Config(cfg.pos @ R.T + np.array([0.3, -1.1, 2.5]), cfg.types, cfg.cell @ R.T)
        out = pot.eval(rc)
        assert out["energy"] == pytest.approx(base["energy"], rel=1e-11)
        np.testing.assert_allclose(out["forces"], base["forces"] @ R.T, rtol=1e-9, atol=1e-9 * np.abs(base["forces"]).max())
        np.testing.assert_allclose(out["virial"], R @ base["virial"] @ R.T, rtol=1e-9,
                                   atol=1e-9 * np.abs(base["virial"]).max())


def test_same_species_permutation_invariance(pot12):
    p, pot = pot12
    cfg = _small_cfg(seed=22, S=2)
    base = pot.eval(cfg)
    perm = np.random.default_rng(0).permutation(cfg.n)
    out = pot.eval(synth.Config(cfg.pos[perm], cfg.types[perm], cfg.cell))
    assert out["energy"] == pytest.approx(base["energy"], rel=1e-12)
    np.testing.assert_allclose(out["forces"], base["forces"][perm], rtol=1e-10, atol=1e-10)


def test_species_relabelling_with_equal_radial_blocks():
    p = _params(10, S=2, seed=4)
    p.c[:] = p.c[0, 0]
    pot = oracle.Potential(p)
    cfg = _small_cfg(seed=23, S=2)
    a = pot.eval(cfg)["energy"]
    b = pot.eval(synth.Config(cfg.pos, 1 - cfg.types, cfg.cell))["energy"]
    assert a == pytest.approx(b, rel=1e-12)


def test_forces_are_finite_differences_and_sum_to_zero(pot12):
    p, pot = pot12
    cfg = _small_cfg(seed=24, S=2)
    base = pot.eval(cfg)
    F = base["forces"]
    rms = np.sqrt(np.mean(F**2))
    assert np.abs(F.sum(0)).max() <= 1e-12 * cfg.n * rms
    h = 1e-5
    for i, k in [(0, 0), (7, 1), (31, 2), (12, 0)]:
        pp = cfg.pos.copy()
        pp[i, k] += h
        pm = cfg.pos.copy()
        pm[i, k] -= h
        fd = -(pot.eval(synth.Config(pp, cfg.types, cfg.cell))["energy"]
               - pot.eval(synth.Config(pm, cfg.types, cfg.cell))["energy"]) / (2 * h)
        assert abs(fd - F[i, k]) <= 1e-7 * rms


def test_virial_is_strain_derivative_and_symmetric(pot12):
    p, pot = pot12
    cfg = _small_cfg(seed=25, S=2)
    W = pot.eval(cfg)["virial"]
    np.testing.assert_allclose(W, W.T, atol=1e-9 * np.abs(W).max())
    h = 1e-6
    for a, b in [(0, 0), (1, 2), (2, 0), (1, 1)]:
        e = np.zeros((3, 3))
        e[a, b] = h
        ep = pot.eval(synth.Config(cfg.pos @ (np.eye(3) + e).T, cfg.types, cfg.cell @ (np.eye(3) + e).T))["energy"]
        em = pot.eval(synth.Config(cfg.pos @ (np.eye(3) - e).T, cfg.types, cfg.cell @ (np.eye(3) - e).T))["energy"]
        fd = -(ep - em) / (2 * h)
        assert abs(fd - W[a, b]) <= 1e-6 * np.abs(W).max()


def test_cutoff_smoothness():
    p = _params(10, S=1, seed=6)
    pot = oracle.Potential(p)
    cell = np.eye(3) * 40.0
    res = []
    for delta in (1e-5, 5e-6, 2.5e-6):
        cfg = synth.Config(np.array([[1.0, 1.0, 1.0], [1.0 + 5.0 - delta, 1.0, 1.0]]), np.zeros(2, np.int32), cell)
        out = pot.eval(cfg)
        res.append((delta, out["energy"], np.abs(out["forces"]).max()))
    for (d1, e1, f1), (d2, e2, f2) in zip(res, res[1:]):
        assert e1 / d1**2 == pytest.approx(e2 / d2**2, rel=2e-3)
        assert f1 / d1 == pytest.approx(f2 / d2, rel=2e-3)
    cfg = synth.Config(np.array([[1.0, 1.0, 1.0], [6.0, 1.0, 1.0]]), np.zeros(2, np.int32), cell)
    out = pot.eval(cfg)
    assert out["energy"] == 0.0 and np.all(out["forces"] == 0.0)


@pytest.mark.parametrize("kind,reps", [("hcp", (1, 1, 1)), ("bcc", (1, 1, 2)), ("fcc", (1, 1, 1))])
def test_extensivity_over_supercells(pot12, kind, reps):
    p, pot = pot12
    rng = np.random.default_rng(3)
    small = synth.perturbed(kind, reps, 0.1, rng, n_species=2)
    base = pot.eval(small)
    big_pos, big_cell = synth.supercell((small.pos @ np.linalg.inv(small.cell), small.cell), (2, 1, 3))
    big = synth.Config(big_pos, np.tile(small.types, 6), big_cell)
    out = pot.eval(big)
    assert out["energy"] == pytest.approx(6 * base["energy"], rel=1e-11)
    np.testing.assert_allclose(out["virial"], 6 * base["virial"], rtol=1e-9, atol=1e-9 * np.abs(base["virial"]).max())


def test_neighbours_equal_independent_brute_force():
    rng = np.random.default_rng(8)
    for kind, reps in [("hcp", (1, 1, 1)), ("bcc", (2, 2, 2)), ("fcc", (1, 2, 1))]:
        cfg = synth.perturbed(kind, reps, 0.2, rng)
        e = rng.uniform(-0.05, 0.05, (3, 3))
        cfg.cell = cfg.cell @ (np.eye(3) + 0.5 * (e + e.T)).T
        counts, j, s, d = oracle.neighbors(cfg.pos, cfg.cell, 5.0)
        got = set()
        q = 0
        for i in range(cfg.n):
            for _ in range(counts[i]):
                got.add((i, int(j[q]), tuple(int(x) for x in s[q])))
                q += 1
        want = set()
        rng_s = range(-4, 5)
        for i in range(cfg.n):
            for jj in range(cfg.n):
                for sv in itertools.product(rng_s, rng_s, rng_s):
                    if jj == i and sv == (0, 0, 0):
                        continue
                    dd = cfg.pos[jj] + np.array(sv) @ cfg.cell - cfg.pos[i]
                    if np.dot(dd, dd) < 25.0:
                        want.add((i, jj, sv))
        assert got == want


def _sampled_cases():
    rng = np.random.default_rng(31)
    one = synth.Config(np.array([[0.3, 0.2, 0.1]]), np.zeros(1, np.int32), np.diag([2.6, 2.9, 3.1]))
    cases = [("one atom, self images", one)]
    for kind, reps, label in (("bcc", (1, 1, 1), "2 atoms, self images"), ("fcc", (1, 1, 2), "8 atoms, self images"),
                              ("hcp", (2, 2, 2), "16 atoms, self images along c"),
                              ("fcc", (2, 2, 2), "32 atoms, no self images")):
        cfg = synth.perturbed(kind, reps, 0.1, rng, n_species=3)
        cases.append((label, cfg))
    return cases


@pytest.mark.parametrize("case", range(5))
def test_sampled_evaluation_equals_full_evaluation(case):
    """The sampled evaluation (used for cells too large for the full oracle) gives the site energies,
    basis rows and forces of the full evaluation, on cells whose atoms see their own periodic images
    (a self-image pair r = s H does not move with the atom and must give no force) and on one
    without."""
    label, cfg = _sampled_cases()[case]
    p = _params(12, S=3, seed=5)
    pot = oracle.Potential(p)
    full = pot.eval(cfg, want_b=True)
    which = np.arange(cfg.n, dtype=np.int32)[::-1].copy()
    smp = pot.eval_sampled(cfg, which)
    scale_f = max(np.abs(full["forces"]).max(), 1e-300)
    np.testing.assert_allclose(smp["site"], full["site"][which], rtol=1e-12, atol=1e-12 * np.abs(full["site"]).max())
    np.testing.assert_allclose(smp["b_atoms"], full["b_atoms"][which], rtol=1e-12,
                               atol=1e-12 * np.abs(full["b_atoms"]).max())
    np.testing.assert_allclose(smp["forces"], full["forces"][which], rtol=0, atol=1e-12 * scale_f, err_msg=label)
    if cfg.n == 1:  # moving the only atom moves every image with it: no force at all
        np.testing.assert_allclose(smp["forces"], 0.0, atol=1e-12 * np.abs(full["site"]).max())


def test_sampled_forces_are_finite_differences():
    """Sampled forces of a 2-atom cell (every neighbour pair of each atom includes images of itself)
    equal central differences of the full energy."""
    rng = np.random.default_rng(8)
    cfg = synth.perturbed("bcc", (1, 1, 1), 0.1, rng, n_species=2)
    pot = oracle.Potential(_params(10, S=2, seed=3))
    smp = pot.eval_sampled(cfg, np.array([0, 1], dtype=np.int32))
    h = 1e-5
    for i in range(2):
        for a in range(3):
            cp, cm = synth.Config(cfg.pos.copy(), cfg.types, cfg.cell), synth.Config(cfg.pos.copy(), cfg.types, cfg.cell)
            cp.pos[i, a] += h
            cm.pos[i, a] -= h
            fd = -(pot.eval(cp)["energy"] - pot.eval(cm)["energy"]) / (2 * h)
            assert abs(smp["forces"][i, a] - fd) <= 1e-6 * max(1.0, np.abs(smp["forces"]).max()), (i, a)
