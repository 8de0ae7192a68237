"""Pins of the relaxation oracle (oracle/relax.py): FIRE reaches the exact minimum of a quadratic;
the cell coordinates driven by the virial reach the minimum of an energy of the cell metric alone
(a closed form for the generalised force on the deformation gradient); positions relax to vanishing
forces at lower energy (a bounded pair energy over the oracle's neighbour lists); a run that
diverges is not reported as converged; the run stops at the first configuration whose grade
reaches gamma_break."""

import numpy as np
import pytest

import oracle
from oracle import relax, selection
from paper_2007_08555_gb300 import codegen, synth


def test_fire_reaches_the_minimum_of_a_quadratic():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.normal(size=(12, 12)))
    K = Q @ np.diag(np.linspace(1.0, 20.0, 12)) @ Q.T
    q_star = rng.normal(size=12)
    q, steps, ok = relax.fire(lambda q: -K @ (q - q_star), np.zeros(12), dt=0.02, dt_max=0.2, fmax=1e-10)
    assert ok and steps < 5000
    np.testing.assert_allclose(q, q_star, atol=1e-9)


def test_cell_relaxes_to_the_metric_minimum():
    # E = kappa/2 |H H^T - G0|_F^2 (no dependence on positions): W = -dE/d(strain) = -2 kappa H^T (G - G0) H
    # with G = H H^T (checked below by central differences); the minimum is any cell with H H^T = G0
    kappa = 0.05
    G0 = np.array([[16.0, 1.0, 0.5], [1.0, 14.0, -0.8], [0.5, -0.8, 18.0]])
    n = 4
    pos = np.random.default_rng(2).uniform(0, 3, size=(n, 3))

    def evaluate(x, H):
        G = H @ H.T
        e = 0.5 * kappa * np.sum((G - G0) ** 2)
        W = -2.0 * kappa * (H.T @ (G - G0) @ H)
        return e, np.zeros_like(x), W

    # the virial formula itself against central differences of the energy under strain
    H = np.eye(3) * 3.7 + 0.2
    _, _, W = evaluate(pos, H)
    h = 1e-6
    for a, b in [(0, 0), (0, 1), (2, 1)]:
        eps = np.zeros((3, 3))
        eps[a, b] = h
        ep = evaluate(pos, H @ (np.eye(3) + eps).T)[0]
        em = evaluate(pos, H @ (np.eye(3) - eps).T)[0]
        assert -(ep - em) / (2 * h) == pytest.approx(W[a, b], rel=1e-6)
    out = relax.relax(evaluate, pos, H, relax_cell=True, fmax=1e-6, smax=1e-9, dt=0.01, dt_max=0.1,
                      max_steps=20000)
    assert out["converged"]
    np.testing.assert_allclose(out["cell"] @ out["cell"].T, G0, atol=1e-5)


@pytest.fixture(scope="module")
def mtp_pot():
    L, S = 8, 2
    labels = synth.labels_from_level_table(codegen.level_table(codegen.build_basis(L)))
    p = synth.scaled_params(L, S, 6, 1.0, 5.0, labels, seed=3, radial_decay=0.5)
    return oracle.Potential(p)


def _lennard_jones(eps=0.1, sigma=2.3, rc=5.0):
    """A bounded pair energy with a smooth cutoff: phi(r) = 4 eps ((s/r)^12 - (s/r)^6) (1 - (r/rc)^2)^2,
    over the oracle's full neighbour lists (each pair twice, hence the 1/2)."""
    def evaluate(x, H):
        counts, j, _, d = oracle.neighbors(x, H, rc)
        i = np.repeat(np.arange(x.shape[0]), counts)
        r = np.linalg.norm(d, axis=1)
        sr6 = (sigma / r) ** 6
        lj, dlj = 4 * eps * (sr6 * sr6 - sr6), 4 * eps * (-12 * sr6 * sr6 + 6 * sr6) / r
        sm, dsm = (1 - (r / rc) ** 2) ** 2, -4 * r / rc**2 * (1 - (r / rc) ** 2)
        phi, dphi = lj * sm, dlj * sm + lj * dsm
        e = 0.5 * phi.sum()
        F = np.zeros_like(x)
        np.add.at(F, i, (dphi / r)[:, None] * d)
        return e, F, np.zeros((3, 3))
    return evaluate


def test_positions_relax_to_vanishing_forces():
    cfg = synth.perturbed("fcc", (2, 2, 2), 0.1, np.random.default_rng(4), n_species=1)
    evaluate = _lennard_jones()
    e0, F0, _ = evaluate(cfg.pos, cfg.cell)
    # the forces are the negative gradient of the energy
    h = 1e-6
    for a, k in [(0, 0), (5, 2)]:
        pp, pm = cfg.pos.copy(), cfg.pos.copy()
        pp[a, k] += h
        pm[a, k] -= h
        assert -(evaluate(pp, cfg.cell)[0] - evaluate(pm, cfg.cell)[0]) / (2 * h) == pytest.approx(F0[a, k], rel=1e-5)
    out = relax.relax(evaluate, cfg.pos, cfg.cell, relax_cell=False, fmax=1e-5, max_steps=5000)
    assert out["converged"] and not out["stopped"]
    e1, F1, _ = evaluate(out["pos"], out["cell"])
    assert np.abs(F1).max() <= 1e-5 < np.abs(F0).max()
    assert e1 < e0
    np.testing.assert_array_equal(out["cell"], cfg.cell)


def test_diverging_run_is_not_converged():
    # an energy without a lower bound: the coordinates run away and the run reports failure
    with np.errstate(over="ignore", invalid="ignore"):
        q, steps, ok = relax.fire(lambda q: q * np.exp(np.minimum(q * q, 700.0)), np.full(3, 0.5), dt=0.5,
                                  dt_max=5.0, max_steps=2000)
    assert not ok


def test_run_stops_at_the_first_extrapolative_configuration(mtp_pot):
    cfg = synth.perturbed("fcc", (2, 2, 2), 0.05, np.random.default_rng(5), n_species=2)
    calls = []

    def evaluate(x, H):
        r = mtp_pot.eval(synth.Config(x, cfg.types, H))
        return r["energy"], r["forces"], r["virial"]

    def grade(x, H):  # a stand-in grade that grows along the trajectory
        calls.append(1)
        return 1.0 + 0.3 * len(calls)

    out = relax.relax(evaluate, cfg.pos, cfg.cell, relax_cell=False, fmax=1e-9, grade=grade, gamma_break=3.0)
    assert out["stopped"] and not out["converged"]
    sel, stop = selection.two_threshold(out["gammas"], 2.0, 3.0)
    assert stop == len(out["gammas"]) - 1 and out["gammas"][-1] >= 3.0
