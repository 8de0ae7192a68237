"""The training optimiser on the GPU (Sec. 2.2) against the oracle's L-BFGS (oracle/train.py).

With the oracle's loss and exact gradient driving oracle/train.py and the library's mtp_train on
the same batch, targets and starting parameters, the losses of the first iterates agree (double
path: the same accepted steps; both take the loss and gradient of the same Eqs. 7, 11, 12), and both
runs drive the loss of a model started near the generating parameters towards zero, for the three
scalings; the float path decreases the loss as well.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import levels, loss as oloss, train
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _case():
    L, S, NQ = 6, 1, 3
    m = len(levels.basis(L))
    pstar = synth.random_params(L, S, NQ, 2.0, 5.0, m, seed=3)
    b = synth.small_cells(n_cfg=6, n_lo=6, n_hi=16, seed=4, max_species=1)
    b.types[:] = 0
    cfgs = [b.config(k) for k in range(b.n_cfg)]
    refs = [oracle.Potential(pstar).eval(c) for c in cfgs]
    theta_star = np.concatenate([pstar.xi, pstar.c.reshape(-1)])
    t0 = theta_star + 1e-3 * np.random.default_rng(5).normal(size=theta_star.size) * np.abs(theta_star)
    return pstar, m, b, cfgs, refs, t0


@pytest.mark.parametrize("scaling", ["molecules", "structures", "vibrations"])
def test_lbfgs_matches_oracle(gpu_lib, scaling):
    pstar, m, b, cfgs, refs, t0 = _case()
    w = (1.0, 0.01, 0.001)
    pot = oracle.Potential(pstar)
    split = lambda t: (t[:m], t[m:].reshape(pstar.c.shape))

    def lg(t):
        xi, c = split(t)
        Lv, gxi, gc = oloss.gradient(pot, cfgs, refs, w, scaling, xi, c)
        return Lv, np.concatenate([gxi, gc.reshape(-1)])

    def lo(t):
        xi, c = split(t)
        return oloss.loss_and_directional(pot, cfgs, refs, w, scaling, xi, c)[0]

    iters = 8
    ref = train.lbfgs(lg, lo, t0, history=5, max_iter=iters, gtol=0.0)
    xi0, c0 = split(t0)
    model = mtp.Model(pstar.lev_max, 1, pstar.n_radial, pstar.r_min, pstar.r_cut, xi0, c0, "fp64")
    e_ref = dev([r["energy"] for r in refs])
    f_ref = dev(np.concatenate([r["forces"] for r in refs]))
    w_ref = dev(np.array([r["virial"].reshape(9) for r in refs]))
    batch = (dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32))
    losses, it, status = model.train(*batch, e_ref, f_ref, w_ref, w, scaling, history=5, max_iter=iters, gtol=0.0)
    assert it == ref["iterations"] and status == 1
    np.testing.assert_allclose(losses, ref["losses"], rtol=1e-6)
    assert losses[-1] < 1e-2 * losses[0]
    # the model holds the final parameters: its loss is the last one
    loss = model.loss(*batch, e_ref, f_ref, w_ref, w, scaling).item()
    assert loss == pytest.approx(losses[-1], rel=1e-12)


def test_float_path_decreases_the_loss(gpu_lib):
    pstar, m, b, cfgs, refs, t0 = _case()
    xi0, c0 = t0[:m], t0[m:].reshape(pstar.c.shape)
    model = mtp.Model(pstar.lev_max, 1, pstar.n_radial, pstar.r_min, pstar.r_cut, xi0, c0, "fp32")
    e_ref = dev([r["energy"] for r in refs])
    f_ref = dev(np.concatenate([r["forces"] for r in refs]))
    w_ref = dev(np.array([r["virial"].reshape(9) for r in refs]))
    batch = (dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32))
    losses, it, status = model.train(*batch, e_ref, f_ref, w_ref, max_iter=20, gtol=0.0)
    assert np.all(np.diff(losses) <= 0) and losses[-1] < 1e-2 * losses[0]
