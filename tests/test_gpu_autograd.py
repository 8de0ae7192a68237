"""The training loss (Sec. 2.2, Eq. 12) as a torch.autograd function of xi and c.

* torch.autograd.gradcheck in double precision on a small case: the library's adjoint (backward,
  which re-evaluates the forces) against torch's central differences of the library's own loss;
* through autograd on the float path, the full 820-entry gradient of the lev_max-20 training loss
  on four cells against the oracle's stored gradient, entry by entry, within 1e-4 of the size of
  the terms each entry sums (the componentwise float bar, tests/test_gpu_full_size.py).
"""

import os
import sys

import numpy as np
import pytest
import torch

import oracle
from oracle import levels
from paper_2007_08555_gb300 import mtp, synth

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_grad_lev20  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _refs(pot, b):
    refs = [pot.eval(b.config(k)) for k in range(b.n_cfg)]
    return (dev([r["energy"] for r in refs]), dev(np.concatenate([r["forces"] for r in refs])),
            dev(np.array([r["virial"].reshape(9) for r in refs])))


def test_gradcheck_double_precision(gpu_lib):
    L, S, NQ = 8, 2, 4
    m = len(levels.basis(L))
    pstar = synth.random_params(L, S, NQ, 2.0, 5.0, m, seed=11)
    p0 = synth.random_params(L, S, NQ, 2.0, 5.0, m, seed=12)
    b = synth.small_cells(n_cfg=3, n_lo=6, n_hi=14, seed=13, max_species=S)
    b.types = np.minimum(b.types, S - 1).astype(np.int32)
    e_ref, f_ref, w_ref = _refs(oracle.Potential(pstar), b)
    model = mtp.Model.from_params(p0, "fp64")
    batch = (dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32))
    xi = dev(p0.xi).requires_grad_(True)
    c = dev(p0.c).requires_grad_(True)
    fn = lambda x, cc: mtp.training_loss(model, x, cc, *batch, e_ref, f_ref, w_ref)
    # dL/dc is summed with double-precision atomics: repeated backward passes agree to rounding only
    # (1e-12 of the gradient's size)
    _, g0, gc0 = model.param_grad(*batch, e_ref, f_ref, w_ref)
    scale = max(float(g0.abs().max()), float(gc0.abs().max()))
    assert torch.autograd.gradcheck(fn, (xi, c), eps=1e-6, atol=1e-7 * scale, rtol=1e-5, nondet_tol=1e-12 * scale)
    loss = fn(xi, c)
    loss.backward()
    _, gxi, gc = model.param_grad(*batch, e_ref, f_ref, w_ref)
    np.testing.assert_allclose(xi.grad.cpu().numpy(), gxi.cpu().numpy(), rtol=1e-12)
    np.testing.assert_allclose(c.grad.cpu().numpy(), gc.cpu().numpy(), rtol=1e-12,
                               atol=1e-14 * np.abs(gc.cpu().numpy()).max())


def test_float_gradient_through_autograd_matches_oracle_entrywise(gpu_lib):
    pstar, p0, b, cells = make_grad_lev20.workload("smooth")  # within float range (see test_gpu_full_size)
    cells_g, _, grad_o, scale_o = make_grad_lev20.read("smooth")
    assert cells_g.tolist() == cells.tolist()
    sub = synth.pack([b.config(int(k)) for k in cells])
    e_ref, f_ref, w_ref = _refs(oracle.Potential(pstar), sub)
    model = mtp.Model.from_params(p0, "fp32")
    batch = (dev(sub.pos), dev(sub.types, torch.int32), dev(sub.cells), dev(sub.cfg_off, torch.int32))
    xi = dev(p0.xi).requires_grad_(True)
    c = dev(p0.c).requires_grad_(True)
    loss = mtp.training_loss(model, xi, c, *batch, e_ref, f_ref, w_ref, make_grad_lev20.WEIGHTS, "vibrations")
    loss.backward()
    g = np.concatenate([xi.grad.cpu().numpy(), c.grad.cpu().numpy().reshape(-1)])
    # parameters that no term reaches (a species pair absent from the cells) must be exactly zero
    zero = scale_o == 0.0
    assert np.all(g[zero] == 0.0)
    worst = np.max(np.abs(g[~zero] - grad_o[~zero]) / scale_o[~zero])
    assert worst <= 1e-4, worst
