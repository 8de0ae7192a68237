"""Pins of the active-selection oracle (oracle/selection.py, Sec. 2.3): hand-worked two-threshold
runs, the determinant lemma for a single swap, dominance and locality of the updated active set,
and the closed-form velocity Verlet trajectory of a harmonic oscillator."""

import itertools

import numpy as np
import pytest

from oracle import maxvol, selection


# -- two thresholds --------------------------------------------------------------------------------
def test_two_threshold_hand_worked():
    # select above 2, stop at the first grade >= 10 (which is selected as well)
    assert selection.two_threshold([0.5, 1.2, 2.5, 1.0, 11.0, 3.0], 2.0, 10.0) == ([2, 4], 4)
    # a grade equal to gamma_select is not selected; no break: the run completes
    assert selection.two_threshold([0.1, 3.0, 2.0], 2.0, 10.0) == ([1], None)
    # equality at gamma_break stops the run
    assert selection.two_threshold([1.0, 10.0, 50.0], 2.0, 10.0) == ([1], 1)
    assert selection.two_threshold([], 1.1, 3.0) == ([], None)
    with pytest.raises(ValueError):
        selection.two_threshold([1.0], 5.0, 5.0)


# -- select-add -------------------------------------------------------------------------------------
def _active(m, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(m, m)) + 3.0 * np.eye(m)


def test_interpolative_candidates_change_nothing():
    m = 6
    A = _active(m, 1)
    rng = np.random.default_rng(2)
    c = rng.uniform(-0.9, 0.9, size=(20, m))  # every |c_j| < 1: gamma < 1
    entered, rows, swaps = selection.select_add(A, c @ A)
    assert entered == [] and swaps == 0 and rows.tolist() == list(range(m))


def test_single_extrapolative_candidate_follows_the_determinant_lemma():
    # b = c A with c_j* = 3 and the rest small: b replaces row j*, and det grows by exactly |c_j*|
    m, jstar = 5, 2
    A = _active(m, 3)
    rng = np.random.default_rng(4)
    pool_c = rng.uniform(-0.5, 0.5, size=(7, m))
    pool_c[4] = rng.uniform(-0.2, 0.2, size=m)
    pool_c[4, jstar] = 3.0
    pool = pool_c @ A
    entered, rows, swaps = selection.select_add(A, pool)
    assert entered == [4] and swaps == 1
    assert rows[jstar] == m + 4 and [r for j, r in enumerate(rows) if j != jstar] == [0, 1, 3, 4]
    stacked = np.vstack([A, pool])
    ratio = abs(np.linalg.det(stacked[rows])) / abs(np.linalg.det(A))
    assert ratio == pytest.approx(3.0, rel=1e-12)


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_updated_active_set_dominates_every_row(seed):
    m = 8
    A = _active(m, seed)
    rng = np.random.default_rng(seed + 100)
    pool = rng.normal(scale=2.0, size=(5 * m, m))
    tol = 1e-3
    entered, rows, _ = selection.select_add(A, pool, tol=tol)
    stacked = np.vstack([A, pool])
    assert len(entered) <= m and len(set(rows.tolist())) == m
    assert maxvol.grades(stacked, stacked[rows]).max() <= 1.0 + tol + 1e-9
    # every swap grows the volume: the update never loses |det A|
    assert abs(np.linalg.det(stacked[rows])) >= abs(np.linalg.det(A))


def test_result_is_a_local_maximum_of_the_volume_brute_force():
    m = 3
    A = _active(m, 8)
    rng = np.random.default_rng(9)
    pool = rng.normal(scale=1.5, size=(5, m))
    stacked = np.vstack([A, pool])
    tol = 1e-3
    _, rows, _ = selection.select_add(A, pool, tol=tol)
    vol = abs(np.linalg.det(stacked[rows]))
    for j, k in itertools.product(range(m), range(len(stacked))):
        if k in rows:
            continue
        trial = rows.copy()
        trial[j] = k
        assert abs(np.linalg.det(stacked[trial])) <= (1.0 + tol) * vol * (1 + 1e-12)


def test_column_scaling_does_not_change_the_choice():
    m = 6
    A = _active(m, 10)
    rng = np.random.default_rng(11)
    pool = rng.normal(scale=2.0, size=(15, m))
    d = np.exp(rng.uniform(-8.0, 8.0, size=m))
    e1, r1, _ = selection.select_add(A, pool)
    e2, r2, _ = selection.select_add(A * d, pool * d)
    assert e1 == e2 and r1.tolist() == r2.tolist()


# -- velocity Verlet with the two-threshold check ---------------------------------------------------
def test_verlet_matches_the_discrete_harmonic_closed_form():
    # x'' = -w^2 x with x(0) = 1, v(0) = 0: velocity Verlet gives x_n = cos(n theta),
    # cos theta = 1 - (w dt)^2 / 2, exactly (the scheme's own recurrence)
    w, dt, n = 1.3, 0.1, 40
    out = selection.velocity_verlet_with_selection(
        lambda x: -w * w * x, lambda x: 0.0, np.array([[1.0, 0.0, 0.0]]), np.zeros((1, 3)), np.array([1.0]),
        dt, n, 1.0, 2.0)
    theta = np.arccos(1.0 - 0.5 * (w * dt) ** 2)
    assert out["stop_step"] is None and out["steps_done"] == n
    assert out["x"][0, 0] == pytest.approx(np.cos(n * theta), abs=1e-12)
    assert out["x"][0, 1:].tolist() == [0.0, 0.0]


def test_selection_along_a_trajectory_follows_the_thresholds():
    w, dt, n = 0.9, 0.2, 60
    grade = lambda x: 1.0 + 4.0 * abs(x[0, 0])  # noqa: E731
    out = selection.velocity_verlet_with_selection(
        lambda x: -w * w * x, grade, np.array([[0.0, 0.0, 0.0]]), np.array([[1.0, 0.0, 0.0]]), np.array([1.0]),
        dt, n, 3.0, 4.5)
    sel_steps, stop = selection.two_threshold(out["gammas"], 3.0, 4.5)
    assert [s for s, _ in out["selected"]] == sel_steps
    assert out["stop_step"] == stop and stop is not None and out["steps_done"] == stop
    # the grade of the stopping configuration is the first to reach the break threshold
    assert out["gammas"][-1] >= 4.5 and max(out["gammas"][:-1]) < 4.5
    assert np.array_equal(out["selected"][-1][1], out["x"])
