"""Oracle: the Jacobian rows of the nonlinear D-optimality criterion (Sec. 2.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper fixes: for a nonlinearly parametrised MTP, linearise the energy in the parameters theta
near their current values; the rows of the tall matrix B become dE(cfg; theta)/dtheta over every
parameter, and the rest of the active-learning algorithm (MaxVol, grades) is unchanged.

Here theta = (xi, c), flattened as [xi (m), c (S, S, N_mu, N_Q) in C order].  E is linear in xi
(Eq. 2), so the first m columns are b(cfg) = sum_i B(n_i); the c columns are the exact
derivatives of E along each unit direction of c (the oracle's forward-mode evaluation).

Reading where the paper is silent: the rows satisfy exact linear relations for every configuration
(Euler's theorem for each radial index mu: scaling the block c[:, :, mu, :] by t scales every
M_{mu, nu} by t, so sum_k c_k dE/dc_k over the block equals sum_alpha n_alpha(mu) xi_alpha b_alpha;
at low levels further relations between the radial blocks), so no m x m submatrix of the full
rows is invertible.  MaxVol therefore runs over a maximal linearly independent set of parameter
columns: those chosen by a QR factorisation with column pivoting of the (column-scaled) training
rows, up to the numerical rank (pivots above 1e-10 of the first), in ascending order.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg


def jacobian_row(pot, cfg, xi, c):
    """dE(cfg)/dtheta as one row [m + c.size]."""
    xi = np.asarray(xi, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    b = pot.eval(cfg, xi=xi, c=c, want_b=True)["b_atoms"].sum(0)
    gc = np.zeros(c.size)
    zero_xi = np.zeros_like(xi)
    for a in range(c.size):
        v = np.zeros(c.size)
        v[a] = 1.0
        gc[a] = pot.eval(cfg, xi=xi, c=c, dxi=zero_xi, dc=v.reshape(c.shape))["d_energy"]
    return np.concatenate([b, gc])


def jacobian_rows(pot, configs, xi, c):
    """The tall matrix B of the nonlinear criterion: one Jacobian row per configuration."""
    return np.array([jacobian_row(pot, cfg, xi, c) for cfg in configs])


def independent_columns(rows, rtol=1e-10):
    """Indices (ascending) of a maximal linearly independent set of the columns of `rows`: the first
    `rank` pivots of a column-pivoted QR of the column-scaled rows, rank = number of |R_kk| above
    rtol |R_00|."""
    R = np.asarray(rows, dtype=np.float64)
    mx = np.abs(R).max(axis=0)
    R = R / np.where(mx > 0, mx, 1.0)
    _, Rq, piv = scipy.linalg.qr(R, pivoting=True, mode="economic")
    d = np.abs(np.diag(Rq))
    rank = int((d > rtol * d[0]).sum())
    return np.sort(piv[:rank])
