"""Oracle: training loss and its exact gradient in theta = {xi, c} (Sec. 2.2, Eqs. 7, 11, 12).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Loss over configurations k with N_k atoms:
    sum_k  s_e(N_k) w_e (E_k - E_k^ref)^2 + s_f(N_k) w_f sum_i |F_ik - F_ik^ref|^2
         + s_s(N_k) w_s |W_k - W_k^ref|_F^2
with the per-configuration scalings of the paper:
    "molecules"  (Eq. 7):  s_e = 1,       s_f = 1,     s_s = 1
    "structures" (Eq. 11): s_e = 1/N^2,   s_f = 1/N,   s_s = 1/N^2
    "vibrations" (Eq. 12): s_e = 1/N,     s_f = 1,     s_s = 1/N
The stress term uses the virial W (extensive, eV): Eq. 11 scales energy and stress by the same
1/N^2, which only keeps both size-independent for an extensive stress measure.

The gradient is exact: the oracle evaluates E, F, W together with their derivatives along one
direction of theta (forward-mode dual numbers), so dL/dtheta . v for a direction v is
    sum_k 2 s_e w_e dE_k (E_k - E^ref) + 2 s_f w_f sum_i dF_ik.(F_ik - F^ref) + 2 s_s w_s dW_k:(W_k - W^ref)
and the full gradient is that product for every unit direction.
"""

from __future__ import annotations

import numpy as np

SCALINGS = {"molecules": 0, "structures": 1, "vibrations": 2}


def scale(kind, n):
    k = SCALINGS[kind] if isinstance(kind, str) else int(kind)
    if k == 0:
        return 1.0, 1.0, 1.0
    if k == 1:
        return 1.0 / n**2, 1.0 / n, 1.0 / n**2
    return 1.0 / n, 1.0, 1.0 / n


def loss_and_directional(pot, configs, refs, weights, kind, xi, c, dxi=None, dc=None):
    """Loss at theta = (xi, c) and, with a direction (dxi, dc), its directional derivative."""
    we, wf, ws = weights
    L = 0.0
    dL = 0.0
    for cfg, ref in zip(configs, refs):
        r = pot.eval(cfg, xi=xi, c=c, dxi=dxi, dc=dc) if dxi is not None else pot.eval(cfg, xi=xi, c=c)
        se, sf, ss = scale(kind, cfg.n)
        de = r["energy"] - ref["energy"]
        dfo = r["forces"] - ref["forces"]
        dw = r["virial"] - ref["virial"]
        L += se * we * de**2 + sf * wf * np.sum(dfo**2) + ss * ws * np.sum(dw**2)
        if dxi is not None:
            dL += (2 * se * we * de * r["d_energy"] + 2 * sf * wf * np.sum(dfo * r["d_forces"])
                   + 2 * ss * ws * np.sum(dw * r["d_virial"]))
    return L, dL


def gradient(pot, configs, refs, weights, kind, xi, c):
    """(loss, dL/dxi [m], dL/dc [S,S,N_mu,N_Q]) by one exact directional derivative per parameter."""
    xi = np.asarray(xi, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    gxi = np.zeros_like(xi)
    gc = np.zeros_like(c)
    L = None
    for a in range(xi.size):
        v = np.zeros_like(xi)
        v[a] = 1.0
        L, gxi[a] = loss_and_directional(pot, configs, refs, weights, kind, xi, c, v, np.zeros_like(c))
    flat = gc.reshape(-1)
    for a in range(flat.size):
        v = np.zeros(flat.size)
        v[a] = 1.0
        L, flat[a] = loss_and_directional(pot, configs, refs, weights, kind, xi, c, np.zeros_like(xi),
                                          v.reshape(c.shape))
    return L, gxi, gc
