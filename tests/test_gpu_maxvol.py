"""GPU parity of the active set (MaxVol) and the extrapolation grade (Sec. 2.3) against the oracle.

* the device MaxVol picks the same rows, in the same positions, with the same number of swaps as
  the oracle on tall matrices with columns spanning nine orders of magnitude;
* on b rows of real configurations (the first 2m of a batch of small cells, lev_max 10 and 16)
  the selection equals the oracle's selection on the oracle's own b rows;
* grades match the oracle within 1e-9 relative; active rows have grade 1; grades from
  mtp_eval_batch equal mtp_grade of its b rows; per-atom grades are the per-atom rows' grades;
* a rank-deficient matrix is reported as MTP_ESINGULAR.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import levels, maxvol
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("K,m,seed", [(40, 9, 1), (232, 116, 2), (60, 17, 3)])
def test_maxvol_matches_oracle_on_scaled_matrices(gpu_lib, K, m, seed):
    L = {9: 8, 116: 16, 17: 10}[m]
    model = mtp.Model.from_params(synth.random_params(L, 1, 4, 2.0, 5.0, m, 0))
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(K, m)) * 10.0 ** np.linspace(-3, 6, m)
    sel_o, swaps_o, g_o = maxvol.maxvol(B)
    sel, swaps, g = model.select_active_set(dev(B))
    assert sel.cpu().numpy().tolist() == sel_o.tolist()
    assert swaps == swaps_o
    assert g <= 1 + 1e-3
    gam = model.grade(dev(B)).cpu().numpy()
    np.testing.assert_allclose(gam, maxvol.grades(B, B[sel_o]), rtol=1e-9)
    np.testing.assert_allclose(gam[sel_o], 1.0, atol=1e-9)
    A, Ai, rows = mtp.mtp_get_active_set(model.h, m)
    np.testing.assert_array_equal(A, B[sel_o])
    # A^-1 A = I up to the conditioning of A (columns spanning nine decades)
    np.testing.assert_allclose((Ai @ A), np.eye(m), atol=1e-5)


@pytest.mark.parametrize("L", [10, 16])
def test_active_set_from_configurations(gpu_lib, L):
    m = len(levels.basis(L))
    p = synth.random_params(L, 3, 8, 2.0, 5.0, m, seed=40 + L)
    b = synth.small_cells(n_cfg=2 * m + 8, n_lo=8, n_hi=48, seed=50 + L)
    model = mtp.Model.from_params(p, "fp64")
    pos, types, cells, off = (dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32))
    out = model.eval_batch(pos, types, cells, off, b_rows=True, b_atoms=True)
    B_gpu = out["b_rows"]
    pot = oracle.Potential(p)
    rows_o = []
    atoms_o = []
    for k in range(b.n_cfg):
        r = pot.eval(b.config(k), want_b=True)
        rows_o.append(r["b_atoms"].sum(0))
        atoms_o.append(r["b_atoms"])
    B_o = np.array(rows_o)
    np.testing.assert_allclose(B_gpu.cpu().numpy(), B_o, rtol=1e-10, atol=1e-12 * np.abs(B_o).max())
    first = 2 * m
    sel_o, swaps_o, _ = maxvol.maxvol(B_o[:first])
    sel, swaps, _ = model.select_active_set(B_gpu[:first].contiguous())
    assert sel.cpu().numpy().tolist() == sel_o.tolist()
    # grades of every configuration, from mtp_grade and from the evaluation itself
    g_ref = maxvol.grades(B_o, B_o[sel_o])
    # grades carry the conditioning of the active-set matrix: forward error ~ cond(A D) * eps
    A_s, _ = maxvol.equilibrate(B_o[sel_o])
    tol = min(1e-3, max(1e-8, 1e-12 * np.linalg.cond(A_s)))  # observed 1.5e-5 at cond 3.6e13
    g = model.grade(B_gpu).cpu().numpy()
    np.testing.assert_allclose(g, g_ref, rtol=tol)
    out2 = model.eval_batch(pos, types, cells, off, grade_cfg=True, grade_atom=True)
    np.testing.assert_allclose(out2["grade_cfg"].cpu().numpy(), g_ref, rtol=tol)
    ga_ref = maxvol.grades(np.concatenate(atoms_o), B_o[sel_o])
    np.testing.assert_allclose(out2["grade_atom"].cpu().numpy(), ga_ref, rtol=tol, atol=tol * np.abs(ga_ref).max())


def test_singular_rows_are_reported(gpu_lib):
    m = 9
    model = mtp.Model.from_params(synth.random_params(8, 1, 4, 2.0, 5.0, m, 0))
    rng = np.random.default_rng(0)
    B = rng.normal(size=(30, m))
    B[:, 4] = 2.0 * B[:, 1]  # rank m - 1
    with pytest.raises(mtp.MTPError) as ei:
        model.select_active_set(dev(B))
    assert ei.value.code == 5
    with pytest.raises(mtp.MTPError) as ei:
        model.grade(dev(B))
    assert ei.value.code == 7
