"""Oracle: the training optimiser (Sec. 2.2: the parameters theta = (xi, c) minimise the loss of
Eqs. 7, 11, 12; the paper names no algorithm).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Reading: limited-memory BFGS (Nocedal and Wright, Numerical Optimization, Algorithm 7.4 and 7.5)
with a backtracking line search on the Armijo condition:
  * direction d = -H g from the two-loop recursion over the last `history` pairs (s, y) with
    s = theta_{k+1} - theta_k, y = g_{k+1} - g_k; initial matrix H0 = (s.y / y.y) I of the newest
    pair, H0 = I / max(1, |g|_inf) before the first pair; a pair with s.y <= 1e-12 |s| |y| is not stored;
  * step t = 1, halved until L(theta + t d) <= L(theta) + 1e-4 t g.d, at most 40 halvings (then the
    run stops, reported as a failed line search);
  * stop when max |g| <= gtol (converged) or after max_iter iterations.
"""

from __future__ import annotations

import numpy as np

C1 = 1e-4
MAX_HALVINGS = 40


def lbfgs(loss_grad, loss, theta0, history=10, max_iter=100, gtol=1e-8):
    """loss_grad(theta) -> (L, g); loss(theta) -> L.  Returns dict(theta, losses, iterations,
    status) with status "converged", "max_iter" or "line_search"; losses[k] is L at iterate k."""
    theta = np.array(theta0, dtype=np.float64)
    L, g = loss_grad(theta)
    S, Y = [], []
    losses = [L]
    for it in range(max_iter):
        if np.abs(g).max() <= gtol:
            return dict(theta=theta, losses=losses, iterations=it, status="converged")
        # two-loop recursion
        q = g.copy()
        alphas = []
        for s, y in reversed(list(zip(S, Y))):
            a = (s @ q) / (y @ s)
            alphas.append(a)
            q = q - a * y
        if S:
            q = q * ((S[-1] @ Y[-1]) / (Y[-1] @ Y[-1]))
        else:
            q = q / max(1.0, float(np.abs(g).max()))
        for (s, y), a in zip(zip(S, Y), reversed(alphas)):
            b = (y @ q) / (y @ s)
            q = q + s * (a - b)
        d = -q
        gd = float(g @ d)
        t = 1.0
        for _ in range(MAX_HALVINGS + 1):
            L_new = loss(theta + t * d)
            if L_new <= L + C1 * t * gd:
                break
            t *= 0.5
        else:
            return dict(theta=theta, losses=losses, iterations=it, status="line_search")
        theta_new = theta + t * d
        L_new, g_new = loss_grad(theta_new)
        s, y = theta_new - theta, g_new - g
        if s @ y > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            S.append(s)
            Y.append(y)
            if len(S) > history:
                S.pop(0)
                Y.pop(0)
        theta, L, g = theta_new, L_new, g_new
        losses.append(L)
    status = "converged" if np.abs(g).max() <= gtol else "max_iter"
    return dict(theta=theta, losses=losses, iterations=max_iter, status=status)
