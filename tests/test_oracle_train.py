"""Pins of the training-optimiser oracle (oracle/train.py, Sec. 2.2): L-BFGS with an Armijo
backtracking line search reaches the exact minimiser of a strictly convex quadratic, decreases the
Rosenbrock function monotonically to its minimum (1, 1), and fits MTP parameters: started near the
parameters that generated the targets, the oracle loss goes to zero."""

import numpy as np

import oracle
from oracle import levels, loss as oloss, train
from paper_2007_08555_gb300 import synth


def test_quadratic_minimum():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.normal(size=(8, 8)))
    K = Q @ np.diag(np.linspace(1.0, 30.0, 8)) @ Q.T
    b = rng.normal(size=8)
    f = lambda x: 0.5 * x @ K @ x - b @ x
    fg = lambda x: (f(x), K @ x - b)
    r = train.lbfgs(fg, f, np.zeros(8), history=8, max_iter=200, gtol=1e-8)
    assert r["status"] == "converged" and r["iterations"] <= 40
    np.testing.assert_allclose(r["theta"], np.linalg.solve(K, b), atol=1e-8)
    assert all(b2 <= b1 + 1e-15 for b1, b2 in zip(r["losses"], r["losses"][1:]))


def test_rosenbrock():
    f = lambda x: (1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2
    g = lambda x: np.array([-2 * (1 - x[0]) - 400 * x[0] * (x[1] - x[0] ** 2), 200 * (x[1] - x[0] ** 2)])
    r = train.lbfgs(lambda x: (f(x), g(x)), f, np.array([-1.2, 1.0]), history=5, max_iter=500, gtol=1e-9)
    assert r["status"] == "converged"
    np.testing.assert_allclose(r["theta"], [1.0, 1.0], atol=1e-7)
    assert all(b2 <= b1 for b1, b2 in zip(r["losses"], r["losses"][1:]))


def test_recovers_generating_parameters():
    L, S, NQ = 6, 1, 3
    m = len(levels.basis(L))
    pstar = synth.random_params(L, S, NQ, 2.0, 5.0, m, seed=3)
    b = synth.small_cells(n_cfg=6, n_lo=6, n_hi=16, seed=4, max_species=1)
    b.types[:] = 0
    cfgs = [b.config(k) for k in range(b.n_cfg)]
    pot = oracle.Potential(pstar)
    refs = [pot.eval(c) for c in cfgs]
    w = (1.0, 0.01, 0.001)
    theta_star = np.concatenate([pstar.xi, pstar.c.reshape(-1)])

    def split(t):
        return t[:m], t[m:].reshape(pstar.c.shape)

    def lg(t):
        xi, c = split(t)
        Lv, gxi, gc = oloss.gradient(pot, cfgs, refs, w, "vibrations", xi, c)
        return Lv, np.concatenate([gxi, gc.reshape(-1)])

    def lo(t):
        xi, c = split(t)
        return oloss.loss_and_directional(pot, cfgs, refs, w, "vibrations", xi, c)[0]

    rng = np.random.default_rng(5)
    t0 = theta_star + 1e-3 * rng.normal(size=theta_star.size) * np.abs(theta_star)
    r = train.lbfgs(lg, lo, t0, history=10, max_iter=60, gtol=1e-12)
    # the loss vanishes at the generating parameters; the parameters themselves are not identifiable
    # (E is unchanged when a radial block c[:, :, mu, :] is scaled by t and each xi_alpha by
    # t^-n_alpha(mu)), so only the loss is checked
    assert r["losses"][-1] <= 1e-7 * r["losses"][0]
    assert all(b2 <= b1 for b1, b2 in zip(r["losses"], r["losses"][1:]))
