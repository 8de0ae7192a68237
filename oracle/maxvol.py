"""Oracle: D-optimality active set, MaxVol and the extrapolation grade (Sec. 2.3, Eq. 13).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper fixes:
  * b_alpha(cfg) = sum_i B_alpha(n_i); the rows b(cfg_k) stack into the tall matrix B (Eq. 13);
  * the active set is the m rows of B whose m x m submatrix A has maximal |det A|;
  * for a row b, c = b A^{-1} and gamma = max_j |c_j|; if gamma > 1 the row replaces row
    argmax_j |c_j| of A and |det A| grows (the MaxVol step, Goreinov et al. 2010);
  * if the active set is also the training set, the fitted xi reproduces the active energies
    and then E(cfg) = sum_j c_j E(cfg_j) for any cfg.  The paper prints xi = (E_1 .. E_m) A^{-1};
    the identity holds for the xi that solves A xi = (E_1 .. E_m)^T, which is how it is read here.

Readings where the paper is silent (each stated in the design notes):
  * start: the m pivot rows of Gaussian elimination with partial pivoting on B;
  * a sweep computes C = B A^{-1} for every row, takes the largest |C_kj| (ties: the first in
    row-major order, i.e. smallest row k, then smallest column j) and swaps while it exceeds
    1 + tol (tol = 1e-3: on real b rows, whose condition number reaches 1e13 even after column
    scaling, the rounding noise of C exceeds 1e-6 and smaller thresholds make the swaps cycle);
  * at most max_iter = 100 m swaps;
  * the columns of B are first scaled by 1 / max |column|: C = B A^{-1} is unchanged by B -> B D
    (it becomes B D (A D)^{-1}), so this only conditions the arithmetic.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg


def b_rows(b_atoms, cfg_off):
    """b(cfg_k) = sum of the per-atom basis rows of the atoms of configuration k (Sec. 2.3)."""
    b_atoms = np.asarray(b_atoms, dtype=np.float64)
    out = np.zeros((len(cfg_off) - 1, b_atoms.shape[1]))
    for k in range(len(cfg_off) - 1):
        out[k] = b_atoms[cfg_off[k]:cfg_off[k + 1]].sum(0)
    return out


def equilibrate(B):
    """Column scaling D = diag(1 / max_r |B_rc|) and B D."""
    B = np.asarray(B, dtype=np.float64)
    mx = np.abs(B).max(axis=0)
    if np.any(mx == 0.0):
        raise np.linalg.LinAlgError("zero column")
    return B / mx, 1.0 / mx


def pivot_rows(B):
    """Row indices chosen as pivots by LU with partial pivoting, in pivot order: B = P L U, and
    row k of P^T B (the k-th pivot row) is row argmax_r P[r, k] of B."""
    B = np.asarray(B, dtype=np.float64)
    m = B.shape[1]
    P, _, _ = scipy.linalg.lu(B)
    return np.asarray([int(np.argmax(P[:, k])) for k in range(m)], dtype=np.int64)


def maxvol(B, tol=1e-3, max_iter=None):
    """Active set of m rows of the tall matrix B.  Returns (rows [m], swaps, final max |C|)."""
    B, _ = equilibrate(B)
    K, m = B.shape
    if K < m:
        raise ValueError("need at least m rows")
    sel = pivot_rows(B)
    _, _, U = scipy.linalg.lu(B)
    if np.any(np.diag(U)[:m] == 0.0):  # an exactly zero pivot; det() would underflow long before
        raise np.linalg.LinAlgError("singular start")
    max_iter = 100 * m if max_iter is None else max_iter
    swaps = 0
    while True:
        C = B @ np.linalg.inv(B[sel])
        flat = int(np.argmax(np.abs(C)))
        k, j = divmod(flat, m)
        g = abs(C[k, j])
        if g <= 1.0 + tol:
            return sel, swaps, g
        if swaps >= max_iter:
            raise RuntimeError("maxvol did not converge")
        sel[j] = k
        swaps += 1


def grades(B_rows, A):
    """gamma = max_j |(b A^{-1})_j| for every row b (Sec. 2.3), evaluated as (b D)(A D)^{-1}."""
    A = np.asarray(A, dtype=np.float64)
    _, d = equilibrate(A)
    C = (np.asarray(B_rows, dtype=np.float64) * d) @ np.linalg.inv(A * d)
    return np.abs(C).max(axis=1)
