"""Pins of the oracle's MaxVol / extrapolation grade (Sec. 2.3) and training loss (Sec. 2.2).

MaxVol, against what the algorithm fixes:
* rows of the active set have c = e_j, so their grade is exactly 1;
* after MaxVol no row of B has |c_j| > 1 + tol (dominance), so no single swap grows |det A|;
* on tiny matrices, brute force over all single swaps confirms a local maximum of |det A|;
* the swap threshold 1 + 1e-3 gives up no |det A| on well-conditioned rows: the selection equals
  the one at 1 + 1e-9;
* grades and the selection are invariant to column scaling of B (A -> A D);
* the interpolation identity: xi with A xi = (E_1..E_m) gives E(cfg) = sum_j c_j E(cfg_j).
Loss:
* its exact directional derivative equals central finite differences in theta (xi and c);
* for w_f = w_s = 0 the xi-gradient has the closed form 2 w_e sum_k s_k (E_k - E_ref) b(cfg_k);
* at targets generated by the oracle at theta*, the gradient vanishes at theta*.
"""

import itertools

import numpy as np
import pytest

import oracle
from oracle import levels, loss, maxvol
from paper_2007_08555_gb300 import synth


def _tall(K, m, seed, scales=None):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(K, m))
    if scales is not None:
        B = B * scales
    return B


def test_pivot_rows_are_textbook_partial_pivoting():
    # the start rows are the pivot rows of Gaussian elimination with partial pivoting, written out
    # here as the textbook loop on small matrices
    for seed in range(4):
        B = _tall(12, 5, seed)
        W = B.copy()
        order = list(range(12))
        for k in range(5):
            p = k + int(np.argmax(np.abs(W[order[k:], k])))
            order[k], order[p] = order[p], order[k]
            for r in order[k + 1:]:
                W[r, k:] -= W[r, k] / W[order[k], k] * W[order[k], k:]
        assert maxvol.pivot_rows(B).tolist() == order[:5]


def test_active_rows_have_unit_grade_and_dominance():
    B = _tall(60, 12, 1, scales=10.0 ** np.linspace(-3, 6, 12))
    sel, swaps, g = maxvol.maxvol(B)
    A = B[sel]
    C = B @ np.linalg.inv(A)
    np.testing.assert_allclose(C[sel], np.eye(12), atol=1e-9)
    assert np.abs(C).max() <= 1 + 1e-3
    gr = maxvol.grades(B, A)
    np.testing.assert_allclose(gr[sel], 1.0, atol=1e-9)
    assert swaps > 0


@pytest.mark.parametrize("K,m,seed", [(34, 17, 1), (200, 17, 2), (232, 116, 3), (500, 60, 5)])
def test_loose_threshold_keeps_the_determinant(K, m, seed):
    # at the end of MaxVol any single swap could raise |det A| by at most 1 + tol; on these rows the
    # threshold of the library (1e-3) and a tight one (1e-9) stop at the same rows
    B = _tall(K, m, seed, scales=10.0 ** np.linspace(-3, 6, m))
    loose, _, _ = maxvol.maxvol(B, tol=1e-3)
    tight, _, g = maxvol.maxvol(B, tol=1e-9)
    assert g <= 1 + 1e-9
    assert loose.tolist() == tight.tolist()
    assert np.linalg.slogdet(B[loose])[1] == np.linalg.slogdet(B[tight])[1]


@pytest.mark.parametrize("K,m,seed", [(6, 2, 0), (8, 3, 1), (10, 4, 2), (9, 2, 3)])
def test_tiny_bruteforce_local_maximum(K, m, seed):
    B = _tall(K, m, seed)
    sel, _, _ = maxvol.maxvol(B)
    d0 = abs(np.linalg.det(B[sel]))
    for pos in range(m):
        for row in range(K):
            if row in sel:
                continue
            s2 = sel.copy()
            s2[pos] = row
            assert abs(np.linalg.det(B[s2])) <= d0 * (1 + 1e-3)
    best = max(abs(np.linalg.det(B[list(c)])) for c in itertools.combinations(range(K), m))
    assert d0 <= best * (1 + 1e-12)
    assert d0 >= best / (m ** (m / 2.0)) * 0.999  # Goreinov-Tyrtyshnikov bound for a dominant submatrix


def test_grade_column_scaling_and_row_order_invariance():
    B = _tall(40, 8, 4)
    sel, _, _ = maxvol.maxvol(B)
    g = maxvol.grades(B, B[sel])
    D = np.diag(10.0 ** np.linspace(-4, 4, 8))
    g2 = maxvol.grades(B @ D, (B @ D)[sel])
    np.testing.assert_allclose(g, g2, rtol=1e-9)
    # the selection with scaled columns is the same (gamma does not see the scaling)
    sel2, _, _ = maxvol.maxvol(B @ D)
    assert sel2.tolist() == sel.tolist()
    # a different row order may end in another local maximum, but it is again dominant
    perm = np.random.default_rng(0).permutation(40)
    sel_p, _, _ = maxvol.maxvol(B[perm])
    assert maxvol.grades(B, B[perm][sel_p]).max() <= 1 + 1e-3


def test_interpolation_identity():
    p = synth.random_params(8, 1, 6, 2.0, 5.0, len(levels.basis(8)), seed=12)
    pot = oracle.Potential(p)
    rng = np.random.default_rng(5)
    cfgs = [synth.random_small_config(rng, 8, 24, max_species=1) for _ in range(30)]
    for c in cfgs:
        c.types[:] = 0
    rows = []
    for c in cfgs:
        rows.append(pot.eval(c, want_b=True)["b_atoms"].sum(0))
    B = np.array(rows)
    # b rows reproduce E exactly: E(cfg) = xi . b(cfg) (Sec. 2.3)
    for c, b in zip(cfgs[:5], B[:5]):
        assert pot.eval(c)["energy"] == pytest.approx(float(p.xi @ b), rel=1e-11)
    sel, _, _ = maxvol.maxvol(B)
    A = B[sel]
    E_active = np.array([pot.eval(cfgs[k])["energy"] for k in sel])
    # Sec. 2.3 prints xi = (E_1 .. E_m) A^{-1}; the identity E(cfg) = sum_j c_j E_j with
    # c = b A^{-1} holds for the xi that fits the active set exactly, A xi = E_active
    xi2 = np.linalg.solve(A, E_active)
    # a potential with xi2 reproduces the active energies and interpolates the rest through c
    C = B @ np.linalg.inv(A)
    for k in range(len(cfgs)):
        e2 = pot.eval(cfgs[k], xi=xi2)["energy"]
        assert e2 == pytest.approx(float(C[k] @ E_active), rel=1e-8, abs=1e-8 * np.abs(E_active).max())


def _loss_setup(L=6, S=2, n_cfg=3, seed=31):
    m = len(levels.basis(L))
    pstar = synth.random_params(L, S, 4, 2.0, 5.0, m, seed=seed)
    p0 = synth.random_params(L, S, 4, 2.0, 5.0, m, seed=seed + 1)
    pot = oracle.Potential(pstar)
    rng = np.random.default_rng(seed)
    cfgs = [synth.random_small_config(rng, 6, 14, max_species=S) for _ in range(n_cfg)]
    for c in cfgs:
        c.types = np.minimum(c.types, S - 1).astype(np.int32)
    refs = [pot.eval(c) for c in cfgs]
    return pot, pstar, p0, cfgs, refs


@pytest.mark.parametrize("kind", ["molecules", "structures", "vibrations"])
def test_loss_directional_derivative_equals_finite_difference(kind):
    pot, pstar, p0, cfgs, refs = _loss_setup()
    rng = np.random.default_rng(2)
    v_xi = rng.normal(size=p0.xi.shape)
    v_c = rng.normal(size=p0.c.shape) * 0.1
    w = (1.0, 0.01, 0.001)
    _, dl = loss.loss_and_directional(pot, cfgs, refs, w, kind, p0.xi, p0.c, v_xi, v_c)
    h = 1e-6
    lp, _ = loss.loss_and_directional(pot, cfgs, refs, w, kind, p0.xi + h * v_xi, p0.c + h * v_c)
    lm, _ = loss.loss_and_directional(pot, cfgs, refs, w, kind, p0.xi - h * v_xi, p0.c - h * v_c)
    assert dl == pytest.approx((lp - lm) / (2 * h), rel=1e-6)


def test_xi_gradient_closed_form_energy_only():
    pot, pstar, p0, cfgs, refs = _loss_setup()
    w = (1.0, 0.0, 0.0)
    L0, gxi, gc = loss.gradient(pot, cfgs, refs, w, "vibrations", p0.xi, p0.c)
    expect = np.zeros_like(p0.xi)
    for c, r in zip(cfgs, refs):
        out = pot.eval(c, xi=p0.xi, c=p0.c, want_b=True)
        expect += 2.0 / c.n * (out["energy"] - r["energy"]) * out["b_atoms"].sum(0)
    np.testing.assert_allclose(gxi, expect, rtol=1e-9)


def test_gradient_vanishes_at_generating_parameters():
    pot, pstar, p0, cfgs, refs = _loss_setup()
    L0, gxi, gc = loss.gradient(pot, cfgs, refs, (1.0, 0.01, 0.001), "vibrations", pstar.xi, pstar.c)
    assert L0 == 0.0
    assert np.abs(gxi).max() == 0.0 and np.abs(gc).max() == 0.0
