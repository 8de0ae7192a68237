"""Active selection on the GPU (Sec. 2.3) against the oracle (oracle/selection.py).

* select-add: the MaxVol update from the current active set picks the same candidates, in the same
  positions, with the same number of swaps as the oracle: interpolative pools change nothing, one
  extrapolative candidate replaces the row its largest |c_j| points at, random pools;
* MD with the two-threshold scheme: the device run selects the same steps, stops at the same step
  and stores the same configurations in its ring buffer as velocity Verlet driven by the oracle's
  forces and grades; thresholds are placed at least 2% away from every grade of the run, and the
  float evaluation with tensor-core grades classifies the steps identically.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import levels, maxvol, selection
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu

MASSES = [26.98, 58.69]
MVV = 103.642696


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _model_with_active_set(L, A):
    m = A.shape[0]
    model = mtp.Model.from_params(synth.random_params(L, 1, 4, 2.0, 5.0, m, 0), "fp64")
    mtp.mtp_set_active_set(model.h, A)
    return model


def _check_against_oracle(L, A, cand):
    entered_o, rows_o, swaps_o = selection.select_add(A, cand)
    model = _model_with_active_set(L, A)
    entered, rows, swaps = model.select_add(dev(cand))
    assert entered == entered_o and rows.tolist() == rows_o.tolist() and swaps == swaps_o
    A_new, _, _ = mtp.mtp_get_active_set(model.h, A.shape[0])
    np.testing.assert_array_equal(A_new, np.vstack([A, cand])[rows_o])
    g = model.grade(dev(np.vstack([A, cand]))).cpu().numpy()
    assert g.max() <= 1 + 1e-3 + 1e-9  # the updated set dominates every row
    return entered


@pytest.mark.parametrize("case", ["interpolative", "single", "random5", "random6", "random7"])
def test_select_add_matches_oracle(gpu_lib, case):
    if case == "interpolative":
        m, L = 9, 8
        A = np.random.default_rng(1).normal(size=(m, m)) + 3.0 * np.eye(m)
        c = np.random.default_rng(2).uniform(-0.9, 0.9, size=(20, m))
        assert _check_against_oracle(L, A, c @ A) == []
    elif case == "single":
        m, L, jstar = 5, 6, 2
        A = np.random.default_rng(3).normal(size=(m, m)) + 3.0 * np.eye(m)
        rng = np.random.default_rng(4)
        pc = rng.uniform(-0.5, 0.5, size=(7, m))
        pc[4] = rng.uniform(-0.2, 0.2, size=m)
        pc[4, jstar] = 3.0
        assert _check_against_oracle(L, A, pc @ A) == [4]
    else:
        seed = int(case[-1])
        m, L = 17, 10
        rng = np.random.default_rng(seed)
        A = rng.normal(size=(m, m)) + 3.0 * np.eye(m)
        cand = rng.normal(size=(30, m)) * 2.5
        _check_against_oracle(L, A, cand)


def _thresholds(gammas):
    """gamma_select and gamma_break between grades of the run, each at least 2% from every grade."""
    g = np.unique(np.asarray(gammas))
    gaps = [(g[k + 1] / g[k], k) for k in range(len(g) - 1) if g[k + 1] > 1.04 * g[k]]
    assert len(gaps) >= 2, g
    ks = sorted(k for _, k in gaps)
    lo = ks[len(ks) // 3]
    hi = ks[(2 * len(ks)) // 3] if ks[(2 * len(ks)) // 3] > lo else ks[-1]
    gs = np.sqrt(g[lo] * g[lo + 1])
    gb = np.sqrt(g[hi] * g[hi + 1])
    assert gs < gb
    return float(gs), float(gb)


@pytest.fixture(scope="module")
def md_case():
    L = 10
    m = len(levels.basis(L))
    p = synth.scaled_params(L, 2, 8, 2.0, 5.0, synth.labels_from_level_table(levels.level_table(L)), seed=31)
    pot = oracle.Potential(p)
    rng = np.random.default_rng(32)
    base = synth.perturbed("fcc", (2, 2, 2), 0.0, rng, n_species=2)
    pool = []
    for k in range(2 * m + 6):
        pool.append(synth.Config(base.pos + rng.normal(0, 0.04, size=base.pos.shape), base.types, base.cell))
    B = np.array([pot.eval(c, want_b=True)["b_atoms"].sum(0) for c in pool])
    sel, _, _ = maxvol.maxvol(B)
    A = B[sel]
    v0 = synth.maxwell_velocities(base.types, MASSES, 1500.0, seed=33)
    mass = np.array(MASSES)[base.types] * MVV
    forces = lambda x: pot.eval(synth.Config(x, base.types, base.cell))["forces"]
    grade = lambda x: maxvol.grades(pot.eval(synth.Config(x, base.types, base.cell), want_b=True)["b_atoms"].sum(0)[None],
                                    A)[0]
    steps = 30
    free = selection.velocity_verlet_with_selection(forces, grade, base.pos, v0, mass, 1.0, steps, 1e299, 1e300)
    gs, gb = _thresholds(free["gammas"])
    run = selection.velocity_verlet_with_selection(forces, grade, base.pos, v0, mass, 1.0, steps, gs, gb)
    return p, base, pool, B, sel, v0, steps, gs, gb, run


@pytest.mark.parametrize("precision", ["fp64", "fp32_tc"])
def test_md_selection_matches_oracle(gpu_lib, md_case, precision):
    p, base, pool, B, sel, v0, steps, gs, gb, run = md_case
    model = mtp.Model.from_params(p, precision)
    model.set_skin(0.3)
    pb = synth.pack(pool)
    rows = mtp.Model.from_params(p, "fp64").eval_batch(dev(pb.pos), dev(pb.types, torch.int32), dev(pb.cells),
                                                       dev(pb.cfg_off, torch.int32), b_rows=True)["b_rows"]
    sel_d, _, _ = model.select_active_set(rows)
    assert sel_d.cpu().tolist() == sel.tolist()
    x, v = dev(base.pos), dev(v0)
    cap = 64
    ring = torch.zeros((cap, base.n, 3), dtype=torch.float64, device="cuda")
    out = model.md_select(x, v, dev(base.types, torch.int32), dev(base.cell), MASSES, 1.0, steps, gs, gb, ring)
    sel_steps = [s for s, _ in run["selected"]]
    assert out["stop_step"] == run["stop_step"]
    assert out["n_selected"] == len(sel_steps) <= cap
    assert out["ring_steps"].tolist() == sel_steps
    tol_x, tol_g = (1e-9, 1e-7) if precision == "fp64" else (1e-4, 1e-3)
    np.testing.assert_allclose(out["gammas"], run["gammas"], rtol=tol_g)
    for q, (_, xs) in enumerate(run["selected"]):
        np.testing.assert_allclose(ring[q].cpu().numpy(), xs, rtol=0, atol=tol_x)
    np.testing.assert_allclose(x.cpu().numpy(), run["x"], rtol=0, atol=tol_x)
