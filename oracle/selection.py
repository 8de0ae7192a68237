"""Oracle: active selection of extrapolative configurations (Sec. 2.3 and the active-learning
iteration that follows it).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper fixes:
  * the extrapolation grade gamma(cfg) = max_j |c_j|, c = b(cfg) A^{-1} (computed by maxvol.grades);
  * the two-threshold scheme: a configuration with gamma > gamma_select is selected for training,
    and the simulation stops at the first configuration with gamma >= gamma_break
    (gamma_select < gamma_break);
  * the update of the active set: MaxVol picks, among the selected (extrapolative) configurations,
    those that enter the active set (the rows that maximise |det A|); at most m of them, however many
    were selected.

Readings where the paper is silent (each stated in the design notes):
  * the configuration that reaches gamma_break is itself selected (its grade exceeds
    gamma_select, since gamma_select < gamma_break);
  * the grade is checked for the configuration at every time step, the starting one included;
  * the update starts MaxVol from the current active set (rows 0 .. m-1 of [A; candidates]) and
    swaps with the rule and tolerance of maxvol.maxvol (largest |C| first, while > 1 + tol); a
    candidate is "selected" if it is in the active set at the end; rows of the old active set may
    leave it.
"""

from __future__ import annotations

import numpy as np

from . import maxvol


def two_threshold(gammas, gamma_select, gamma_break):
    """Steps selected along a run with grades `gammas` (one per step, in order) and the step at
    which the run stops (None if it completes).  Selected: gamma > gamma_select, up to and including
    the stopping step; stopping step: the first with gamma >= gamma_break."""
    if not gamma_select < gamma_break:
        raise ValueError("need gamma_select < gamma_break")
    selected = []
    for t, g in enumerate(gammas):
        if g > gamma_select:
            selected.append(t)
        if g >= gamma_break:
            return selected, t
    return selected, None


def select_add(A, candidates, tol=1e-3, max_iter=None):
    """New active set from the current one (rows of A, m x m) and candidate rows (K x m).

    Returns (entered, rows, swaps): the candidate indices in the final active set (ascending),
    the final active set as indices into the stacked matrix [A; candidates] (position j = row j of
    the new A) and the number of swaps."""
    A = np.asarray(A, dtype=np.float64)
    cand = np.asarray(candidates, dtype=np.float64).reshape(-1, A.shape[1])
    m = A.shape[0]
    if A.shape != (m, m):
        raise ValueError("A must be square")
    B, _ = maxvol.equilibrate(np.vstack([A, cand]))  # column scaling leaves C = B A^{-1} unchanged
    sel = np.arange(m)
    max_iter = 100 * m if max_iter is None else max_iter
    swaps = 0
    while True:
        C = B @ np.linalg.inv(B[sel])
        flat = int(np.argmax(np.abs(C)))
        k, j = divmod(flat, m)
        if abs(C[k, j]) <= 1.0 + tol:
            break
        if swaps >= max_iter:
            raise RuntimeError("select_add did not converge")
        sel[j] = k
        swaps += 1
    entered = sorted(int(k - m) for k in sel if k >= m)
    return entered, sel, swaps


def velocity_verlet_with_selection(forces, grade, x0, v0, masses, dt, n_steps, gamma_select, gamma_break):
    """Velocity Verlet (half kick v += F/(2M) dt, drift x += v dt, half kick with the new forces) with
    the two-threshold check of every configuration, the starting one included.  Consistent units:
    the caller scales `masses` so that F / M dt is a velocity.

    forces(x) -> F [N, 3]; grade(x) -> gamma.  Returns dict(x, v, steps_done, selected (list of
    (step, x copy)), stop_step, gammas)."""
    x = np.array(x0, dtype=np.float64)
    v = np.array(v0, dtype=np.float64)
    inv_m = 1.0 / np.asarray(masses, dtype=np.float64)[:, None]
    gammas = []
    selected = []
    F = forces(x)
    step = 0
    while True:
        g = float(grade(x))
        gammas.append(g)
        if g > gamma_select:
            selected.append((step, x.copy()))
        if g >= gamma_break:
            return dict(x=x, v=v, steps_done=step, selected=selected, stop_step=step, gammas=gammas)
        if step == n_steps:
            return dict(x=x, v=v, steps_done=step, selected=selected, stop_step=None, gammas=gammas)
        v = v + 0.5 * dt * F * inv_m
        x = x + dt * v
        F = forces(x)
        v = v + 0.5 * dt * F * inv_m
        step += 1
