"""Pins of the nonlinear-criterion oracle (oracle/nonlinear.py, Sec. 2.3): the Jacobian row of a
configuration is the derivative of its energy in every parameter, checked by central differences
of the oracle's energy; its xi part is the linear row b(cfg) and its c part obeys Euler's theorem
for the homogeneous terms of E."""

import numpy as np
import pytest

import oracle
from oracle import levels, nonlinear
from paper_2007_08555_gb300 import codegen, synth


@pytest.fixture(scope="module")
def setup():
    L, S, NQ = 6, 2, 3
    m = codegen.build_basis(L).m
    p = synth.random_params(L, S, NQ, 2.0, 5.0, m, seed=4)
    rng = np.random.default_rng(5)
    configs = [synth.perturbed("fcc", (2, 2, 2), 0.1, rng, n_species=S) for _ in range(2)]
    return p, oracle.Potential(p), configs


def test_row_matches_central_differences_of_the_energy(setup):
    p, pot, configs = setup
    cfg = configs[0]
    row = nonlinear.jacobian_row(pot, cfg, p.xi, p.c)
    m = p.xi.size
    theta = np.concatenate([p.xi, p.c.reshape(-1)])

    def energy(t):
        return pot.eval(cfg, xi=t[:m], c=t[m:].reshape(p.c.shape))["energy"]

    rng = np.random.default_rng(6)
    for a in list(rng.choice(m, 3, replace=False)) + list(m + rng.choice(p.c.size, 6, replace=False)):
        h = 1e-4 * max(1.0, abs(theta[a]))
        tp, tm = theta.copy(), theta.copy()
        tp[a] += h
        tm[a] -= h
        num = (energy(tp) - energy(tm)) / (2 * h)
        assert row[a] == pytest.approx(num, rel=1e-6, abs=1e-9 * np.abs(row).max()), a


def test_xi_part_is_the_linear_row(setup):
    p, pot, configs = setup
    for cfg in configs:
        row = nonlinear.jacobian_row(pot, cfg, p.xi, p.c)
        b = pot.eval(cfg, want_b=True)["b_atoms"].sum(0)
        np.testing.assert_array_equal(row[:p.xi.size], b)
        # E is linear in xi: E = xi . b
        assert float(p.xi @ b) == pytest.approx(pot.eval(cfg)["energy"], rel=1e-12)


def test_c_part_satisfies_euler_homogeneity(setup):
    # B_alpha is a product of n_alpha moments, each linear in c (Eqs. 3, 5), so
    # c . dE/dc = sum_alpha n_alpha xi_alpha B_alpha (Euler's theorem, term by term)
    p, pot, configs = setup
    L = p.lev_max
    comps = levels.connected_components(L)
    n_alpha = np.array([sum(comps[k].n for k in b.components) for b in levels.basis(L)])
    for cfg in configs:
        row = nonlinear.jacobian_row(pot, cfg, p.xi, p.c)
        b = pot.eval(cfg, want_b=True)["b_atoms"].sum(0)
        m = p.xi.size
        lhs = float(p.c.reshape(-1) @ row[m:])
        rhs = float(np.sum(n_alpha * p.xi * b))
        assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-12 * np.abs(p.xi * b).sum())


def test_rows_satisfy_euler_per_radial_index_and_independent_columns_span_them():
    """Every Jacobian row satisfies, for each radial index mu, sum over the block c[:, :, mu, :] of
    c_k dE/dc_k = sum_alpha n_alpha(mu) xi_alpha b_alpha (Euler's theorem for the block scaling);
    the independent columns drop at least one column per mu, are of full rank, and reproduce every
    dropped column by least squares."""
    L, S, NQ = 8, 2, 4
    p = synth.random_params(L, S, NQ, 2.0, 5.0, len(levels.basis(L)), seed=31)
    b = synth.small_cells(n_cfg=60, n_lo=6, n_hi=24, seed=32, max_species=S)
    b.types = np.minimum(b.types, S - 1).astype(np.int32)
    rows = nonlinear.jacobian_rows(oracle.Potential(p), [b.config(k) for k in range(b.n_cfg)], p.xi, p.c)
    m = len(p.xi)
    labels = synth.labels_from_level_table(levels.level_table(L))
    n_mu = p.c.shape[2]
    for mu in range(n_mu):
        mask = np.zeros(p.c.shape)
        mask[:, :, mu, :] = 1.0
        nmu = np.array([sum(1 for (mm, _) in lab if mm == mu) for lab in labels])
        lhs = rows[:, m:] @ (p.c * mask).reshape(-1)
        rhs = rows[:, :m] @ (nmu * p.xi)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-12 * np.abs(rhs).max())
    cols = nonlinear.independent_columns(rows)
    w = rows.shape[1]
    assert len(cols) <= w - n_mu and np.all(np.diff(cols) > 0)
    kept = rows[:, cols] / np.abs(rows[:, cols]).max(0)
    sv = np.linalg.svd(kept, compute_uv=False)
    assert sv[-1] > 1e-9 * sv[0]
    dropped = [k for k in range(w) if k not in set(cols.tolist())]
    coef, *_ = np.linalg.lstsq(rows[:, cols], rows[:, dropped], rcond=None)
    resid = np.abs(rows[:, cols] @ coef - rows[:, dropped]).max(0) / np.abs(rows[:, dropped]).max(0)
    assert resid.max() <= 1e-8
