"""Oracle: structure relaxation with early stop on extrapolation (the relaxation of the paper's
convex-hull example: energy minimisation over atomic positions and lattice vectors, ending either
relaxed or at the first extrapolative configuration).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper fixes what is minimised (the potential energy, over positions and lattice vectors), the
end states (practically zero forces and stresses, or an extrapolative configuration, i.e. grade
>= gamma_break) and that the trajectory is what active selection inspects.  It does not name the
minimiser.  Readings (each stated in the design notes):
  * the minimiser is FIRE (Bitzek, Koskinen, Gahler, Moseler, Gumbsch, Phys. Rev. Lett. 97,
    170201 (2006)): semi-implicit Euler steps with unit masses, the velocity mixed towards the
    force direction v <- (1 - a) v + a |v| F/|F|, and after N_min steps with P = F.v > 0 the step
    grows (dt <- min(f_inc dt, dt_max)) and a shrinks (a <- f_a a); when P <= 0 the velocity is
    zeroed, dt <- f_dec dt and a <- a_start.  Constants: N_min 5, f_inc 1.1, f_dec 0.5,
    a_start 0.1, f_a 0.99;
  * the cell enters through the deformation gradient D of the starting cell (cell rows H = H0 D^T,
    positions x = u D^T with u in the starting frame); the force on u is F D and the force on D is
    W D^{-T} / scale, with W = -dE/d(strain) the virial (eV) and scale the number of atoms, so that
    cell and atom coordinates move at comparable rates;
  * converged when max_i |F_i| <= fmax and max |W| / volume <= smax; the grade is checked for every
    configuration of the trajectory, the starting one included.
"""

from __future__ import annotations

import numpy as np

N_MIN, F_INC, F_DEC, A_START, F_A = 5, 1.1, 0.5, 0.1, 0.99


def fire(grad_force, q0, dt=0.1, dt_max=1.0, fmax=1e-6, max_steps=10000, converged=None):
    """FIRE minimisation of a function with force -grad = grad_force(q) over a flat vector q.
    converged(q, f) -> bool overrides the default max |f| <= fmax test.  Returns (q, steps, ok);
    ok is False when the step limit is reached or q or the force stops being finite."""
    q = np.array(q0, dtype=np.float64)
    v = np.zeros_like(q)
    a = A_START
    n_pos = 0
    for step in range(max_steps + 1):
        f = grad_force(q)
        if not (np.all(np.isfinite(q)) and np.all(np.isfinite(f))):
            return q, step, False  # diverged
        done = converged(q, f) if converged is not None else np.abs(f).max() <= fmax
        if done:
            return q, step, True
        if step == max_steps:
            break
        P = float(f @ v)
        if P > 0.0:
            fn = np.linalg.norm(f)
            v = (1.0 - a) * v + a * np.linalg.norm(v) * f / fn
            n_pos += 1
            if n_pos > N_MIN:
                dt = min(dt * F_INC, dt_max)
                a *= F_A
        else:
            v[:] = 0.0
            dt *= F_DEC
            a = A_START
            n_pos = 0
        v = v + dt * f  # semi-implicit Euler, unit masses
        q = q + dt * v
    return q, max_steps, False


def relax(evaluate, pos, cell, relax_cell=True, fmax=1e-4, smax=1e-5, grade=None, gamma_break=np.inf,
          dt=0.05, dt_max=0.5, max_steps=5000):
    """Relax positions (and the cell) of one configuration.

    evaluate(pos, cell) -> (energy, forces [N, 3], virial [3, 3]); grade(pos, cell) -> gamma or None.
    Returns dict(pos, cell, energy, steps, converged, stopped (extrapolation), gammas)."""
    pos0 = np.asarray(pos, dtype=np.float64)
    H0 = np.asarray(cell, dtype=np.float64)
    n = pos0.shape[0]
    state = {"gammas": [], "stopped": False}

    def unpack(q):
        u = q[:3 * n].reshape(n, 3)
        D = q[3 * n:].reshape(3, 3) if relax_cell else np.eye(3)
        return u @ D.T, H0 @ D.T, D

    def forces(q):
        x, H, D = unpack(q)
        e, F, W = evaluate(x, H)
        state["last"] = (e, F, W, x, H)
        if grade is not None:
            g = float(grade(x, H))
            state["gammas"].append(g)
            if g >= gamma_break:
                state["stopped"] = True
        fu = F @ D
        if not relax_cell:
            return fu.reshape(-1)
        fD = W @ np.linalg.inv(D).T / n
        return np.concatenate([fu.reshape(-1), fD.reshape(-1)])

    def converged(q, f):
        if state["stopped"]:
            return True
        e, F, W, x, H = state["last"]
        ok = np.abs(F).max() <= fmax
        if relax_cell:
            ok = ok and np.abs(W).max() / abs(np.linalg.det(H)) <= smax
        return ok

    q0 = pos0.reshape(-1)
    if relax_cell:
        q0 = np.concatenate([q0, np.eye(3).reshape(-1)])
    q, steps, ok = fire(forces, q0, dt=dt, dt_max=dt_max, max_steps=max_steps, converged=converged)
    x, H, _ = unpack(q)
    e = state["last"][0]
    return dict(pos=x, cell=H, energy=e, steps=steps, converged=ok and not state["stopped"],
                stopped=state["stopped"], gammas=state["gammas"])
