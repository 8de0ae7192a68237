"""The nonlinear extrapolation criterion on the GPU (Sec. 2.3) against the oracle (oracle/nonlinear.py).

* Jacobian rows dE(cfg)/dtheta = [b(cfg), dE/dc] of a batch of small cells equal the oracle's rows
  (forward-mode derivatives of E along every unit direction of c): 1e-9 relative in double precision,
  1e-4 of each row's norm in float;
* with the nonlinear kind over the oracle's independent parameter columns (the full rows obey Euler's
  theorem per radial block and are rank-deficient), MaxVol over the first 2 w rows picks the oracle's
  active set, and the grades of every row match the oracle's within the conditioning bound of
  tests/test_gpu_maxvol.py; grade requests of mtp_eval_batch are refused; a model file keeps the
  nonlinear active set bit for bit.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import levels, maxvol, nonlinear
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _case(n_cfg, seed):
    L, S, NQ = 8, 2, 4
    p = synth.random_params(L, S, NQ, 2.0, 5.0, len(levels.basis(L)), seed=seed)
    b = synth.small_cells(n_cfg=n_cfg, n_lo=6, n_hi=24, seed=seed + 1, max_species=S)
    b.types = np.minimum(b.types, S - 1).astype(np.int32)
    return p, b


def _batch(b):
    return dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_jacobian_rows_match_oracle(gpu_lib, precision):
    p, b = _case(6, 21)
    rows_o = nonlinear.jacobian_rows(oracle.Potential(p), [b.config(k) for k in range(b.n_cfg)], p.xi, p.c)
    model = mtp.Model.from_params(p, precision)
    rows = model.jacobian_rows(*_batch(b)).cpu().numpy()
    assert rows.shape == rows_o.shape == (b.n_cfg, model.m + p.c.size)
    if precision == "fp64":
        np.testing.assert_allclose(rows, rows_o, rtol=1e-9, atol=1e-12 * np.abs(rows_o).max())
    else:
        err = np.linalg.norm(rows - rows_o, axis=1) / np.linalg.norm(rows_o, axis=1)
        assert err.max() <= 1e-4, err.max()


def test_nonlinear_active_set_and_grades(gpu_lib, tmp_path):
    p, b = _case(100, 31)
    pot = oracle.Potential(p)
    full_o = nonlinear.jacobian_rows(pot, [b.config(k) for k in range(b.n_cfg)], p.xi, p.c)
    cols = nonlinear.independent_columns(full_o)  # the full rows are rank-deficient (Euler)
    rows_o = full_o[:, cols]
    model = mtp.Model.from_params(p, "fp64")
    model.set_grade_kind(1, cols)
    w = model.grade_width
    assert w == len(cols) < model.m + p.c.size and 2 * w <= b.n_cfg
    rows = model.jacobian_rows(*_batch(b))
    assert rows.shape == (b.n_cfg, w)
    sel_o, swaps_o, _ = maxvol.maxvol(rows_o[:2 * w])
    sel, swaps, _ = model.select_active_set(rows[:2 * w].contiguous())
    assert sel.cpu().numpy().tolist() == sel_o.tolist() and swaps == swaps_o
    g_ref = maxvol.grades(rows_o, rows_o[sel_o])
    A_s, _ = maxvol.equilibrate(rows_o[sel_o])
    tol = min(1e-3, max(1e-8, 1e-12 * np.linalg.cond(A_s)))
    g = model.grade(rows).cpu().numpy()
    np.testing.assert_allclose(g, g_ref, rtol=tol)
    with pytest.raises(mtp.MTPError) as ei:
        model.eval_batch(*_batch(b), grade_cfg=True)
    assert ei.value.code == 8
    path = str(tmp_path / "nonlinear.mtp")
    model.save(path)
    again = mtp.Model.load(path)
    assert again.grade_width == w
    np.testing.assert_array_equal(again.grade(rows).cpu().numpy(), g)
