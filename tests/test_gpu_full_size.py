"""GPU parity at the stated sizes of the batched, gradient and large-cell workloads.

* 4096 cells of 8-256 atoms, 1-3 species, lev_max 16 (303,192 atoms): energy, forces and virial of
  every cell against the oracle at the FP64 and FP32 bars (the float energy against the atoms'
  energy scale sum_i |V_i|; cells with a pair below R_min, where the Chebyshev basis is evaluated
  outside [-1, 1], at twice the float bars); b rows; the active set chosen by MaxVol
  over the first 2m cells equals the oracle's; the grade of every cell (Sec. 2.3) within the
  first-order bound that the accuracy of its inputs allows (below).
* the lev_max-20 training loss (Sec. 2.2, Eq. 12): the full 820-entry gradient on four cells against
  the oracle's stored gradient, entry by entry; four random projections of the gradient on all 2048
  cells.  The double path on the stated recipe (R_min 2, c ~ N(0, 0.1), scaled xi) and on the smooth
  one (R_min 1, c damped by 0.5^b); the float path on the smooth one, since on the stated recipe the
  gradient leaves the float range (1e57 in double precision over the 2048 cells).
* the 1,048,576-atom ternary fcc cell at lev_max 20 on the stated recipe: site energies, basis rows
  and forces of 256 sampled atoms against the oracle's sampled evaluation; E = sum of site
  energies; forces sum to zero.

Grade bound: gamma = max_j |(b A^-1)_j|.  Inputs b and A known to relative accuracies d_b and d_A
move c = b A^-1 by at most  d_b (|b| |A^-1|)_j + d_A (|c| |A| |A^-1|)_j  (first order), so a grade
is checked against  max_j of that  (plus 1e-12 gamma).  The oracle's A, b and A^-1 give the bound.

Gradient bound (float path): entry a of dL/dtheta sums terms 2 s w (q - q_ref) dq/da over
energies, force components and virial components; each q and dq/da of the float path is within
the float bar (1e-4 relative, the loosest of the energy, force and virial bars) of the exact value,
so the entry is within 1e-4 of the sum of the absolute values of its terms (the stored scale).
Where that scale is not available (projections over all 2048 cells) the same bar is applied
normwise: |g_float - g| <= 1e-4 |g|.
"""

import os
import sys

import numpy as np
import pytest
import torch

import oracle
from oracle import levels, loss as oloss, maxvol
from paper_2007_08555_gb300 import mtp, synth

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_grad_lev20  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(e=1e-10, f=1e-10, w=1e-10, b=1e-10), "fp32": dict(e=1e-5, f=1e-4, w=1e-4, b=1e-4)}


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def grade_bound(B, A, d_b, d_A):
    """First-order bound on the change of gamma = max_j |(b A^-1)_j| when b and A move by the
    relative amounts d_b and d_A (entrywise)."""
    Ai = np.linalg.inv(A * (1.0 / np.abs(A).max(0))) * (1.0 / np.abs(A).max(0))[:, None]
    C = B @ Ai
    t = d_b * (np.abs(B) @ np.abs(Ai)) + d_A * ((np.abs(C) @ np.abs(A)) @ np.abs(Ai))
    return t.max(axis=1)


# ---------------------------------------------------------------------------------------------
# 4096 cells, lev_max 16
# ---------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def batch4096():
    b = synth.small_cells(n_cfg=4096, seed=3)
    m = len(levels.basis(16))
    p = synth.random_params(16, 3, 8, 2.0, 5.0, m, seed=3)
    pot = oracle.Potential(p)
    E, W, B = np.zeros(b.n_cfg), np.zeros((b.n_cfg, 9)), np.zeros((b.n_cfg, m))
    F = np.zeros((b.n_atoms, 3))
    sabs = np.zeros(b.n_cfg)  # sum of |site energies|: the size of the terms each E sums
    rmin = np.zeros(b.n_cfg)  # shortest pair distance of each cell
    for k in range(b.n_cfg):
        c = b.config(k)
        r = pot.eval(c, want_b=True)
        a0, a1 = b.cfg_off[k], b.cfg_off[k + 1]
        E[k], W[k], B[k], F[a0:a1] = r["energy"], r["virial"].reshape(9), r["b_atoms"].sum(0), r["forces"]
        sabs[k] = np.abs(r["site"]).sum()
        d = oracle.neighbors(c.pos, c.cell, 5.0)[3]
        rmin[k] = np.linalg.norm(d, axis=1).min() if len(d) else np.inf
    return b, p, m, E, F, W, B, sabs, rmin


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_config3_batch4096_lev16(gpu_lib, batch4096, precision):
    b, p, m, E, F, W, B, sabs, rmin = batch4096
    assert b.n_cfg == 4096 and b.n_atoms > 250_000
    pos, types, cells, off = dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32)
    model = mtp.Model.from_params(p, precision)
    out = model.eval_batch(pos, types, cells, off, b_rows=True)
    e, f = out["energy"].cpu().numpy(), out["forces"].cpu().numpy()
    w, br = out["virial"].cpu().numpy().reshape(-1, 9), out["b_rows"].cpu().numpy()
    tol = TOL[precision]
    n = np.diff(b.cfg_off)
    # energy: relative to |E| on the double path; on the float path relative to the energy scale of
    # the atoms, sum_i |V_i| >= |E| (a float sum of per-atom terms that cancel cannot hold 1e-5 of |E|:
    # this recipe has cells with sum |V_i| / |E| up to 1.4e3)
    escale = np.abs(E) if precision == "fp64" else sabs
    re = np.abs(e - E) / np.maximum(escale, 1e-300)
    rf, rw, rb = np.zeros(b.n_cfg), np.zeros(b.n_cfg), np.zeros(b.n_cfg)
    for k in range(b.n_cfg):
        a0, a1 = b.cfg_off[k], b.cfg_off[k + 1]
        rms = np.sqrt(np.mean(F[a0:a1] ** 2))
        rf[k] = np.sqrt(np.mean((f[a0:a1] - F[a0:a1]) ** 2)) / max(rms, 1e-300)
        rw[k], rb[k] = rel(w[k], W[k]), rel(br[k], B[k])
    # float path: cells with a pair below R_min evaluate the Chebyshev basis outside [-1, 1], where its
    # growth (energies up to 5e9 eV/atom in this recipe) amplifies float rounding to about 1e-5 of
    # the energy; they are held to twice the bars, all other cells to the bars
    deep = (rmin < p.r_min) if precision == "fp32" else np.zeros(b.n_cfg, bool)
    scale = np.where(deep, 2.0, 1.0)
    bad = np.nonzero((re > tol["e"] * scale) | (rf > tol["f"] * scale) | (rw > tol["w"] * scale) |
                     (rb > tol["b"] * scale))[0]
    print(f"{precision}: {int(deep.sum())} cells with a pair below R_min; worst rel E {re.max():.2e} "
          f"(others {re[~deep].max() if (~deep).any() else 0.0:.2e})")
    rmin_bad = [float(rmin[k]) for k in bad[:8]]
    assert len(bad) == 0, (f"{len(bad)} cells outside the bars; worst rel E {re.max():.2e} F {rf.max():.2e} "
                           f"W {rw.max():.2e} b {rb.max():.2e}; first: " +
                           "; ".join(f"cfg {k}: n {n[k]} E/n {E[k] / n[k]:.3e} sum|V|/|E| {sabs[k] / abs(E[k]):.2e} "
                                     f"relE {re[k]:.2e} relF {rf[k]:.2e} relW {rw[k]:.2e} relb {rb[k]:.2e} "
                                     f"r_min {rm:.3f}" for k, rm in zip(bad[:8], rmin_bad)))
    # active set over the first 2m cells (the oracle's MaxVol on the oracle's rows)
    sel_o, _, _ = maxvol.maxvol(B[:2 * m])
    A = B[sel_o]
    g_ref = maxvol.grades(B, A)
    if precision == "fp64":
        sel, _, _ = model.select_active_set(out["b_rows"][:2 * m].contiguous())
        assert sel.cpu().numpy().tolist() == sel_o.tolist()
        d_A = tol["b"]
    else:  # the float model grades against the double-precision active set of the oracle's rows
        mtp.mtp_set_active_set(model.h, A)
        d_A = 0.0
    out = model.eval_batch(pos, types, cells, off, grade_cfg=True)
    g = out["grade_cfg"].cpu().numpy()
    bound = grade_bound(B, A, tol["b"], d_A) + 1e-12 * g_ref
    assert np.all(np.abs(g - g_ref) <= bound), float(np.max(np.abs(g - g_ref) / bound))
    assert np.all(np.abs(g[sel_o] - 1.0) <= bound[sel_o])


# ---------------------------------------------------------------------------------------------
# training-loss gradient, lev_max 20, stated recipe
# ---------------------------------------------------------------------------------------------
W8 = make_grad_lev20.WEIGHTS


def _batch_tensors(b):
    return dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32)


def _targets(pot, cfgs):
    refs = [pot.eval(c) for c in cfgs]
    return (refs, np.array([r["energy"] for r in refs]), np.concatenate([r["forces"] for r in refs]),
            np.array([r["virial"].reshape(9) for r in refs]))


# The float path runs on the smooth recipe: on the stated one the lev_max-20 gradient leaves the float
# range (1e57 over the 2048 cells in double precision), so only the double path is checked there.
@pytest.mark.parametrize("precision,recipe", [("fp64", "stated"), ("fp64", "smooth"), ("fp32", "smooth")])
def test_config4_gradient_entrywise_four_cells(gpu_lib, precision, recipe):
    pstar, p0, b, cells = make_grad_lev20.workload(recipe)
    cells_g, loss_o, grad_o, scale_o = make_grad_lev20.read(recipe)
    assert cells_g.tolist() == cells.tolist()
    cfgs = [b.config(int(k)) for k in cells]
    sub = synth.pack(cfgs)
    refs, e_ref, f_ref, w_ref = _targets(oracle.Potential(pstar), cfgs)
    model = mtp.Model.from_params(p0, precision)
    loss, dxi, dc = (t.cpu().numpy() for t in model.param_grad(*_batch_tensors(sub), dev(e_ref), dev(f_ref),
                                                                 dev(w_ref), W8, "vibrations"))
    g = np.concatenate([dxi, dc.reshape(-1)])
    assert g.shape == grad_o.shape == (820,)
    if precision == "fp64":
        assert loss[0] == pytest.approx(loss_o, rel=1e-10)
        assert np.all(np.abs(g - grad_o) <= 1e-8 * np.abs(grad_o) + 1e-10 * scale_o)
    else:
        # loss: first-order bound from the float bars on E, F, W at theta_0 (oracle values)
        now = [oracle.Potential(p0).eval(c) for c in cfgs]
        lb = 0.0
        for c, r, q in zip(cfgs, refs, now):
            se, sf, ss = oloss.scale("vibrations", c.n)
            lb += 2 * W8[0] * se * abs(q["energy"] - r["energy"]) * 1e-5 * abs(q["energy"])
            lb += 2 * W8[1] * sf * np.linalg.norm(q["forces"] - r["forces"]) * 1e-4 * np.linalg.norm(q["forces"])
            lb += 2 * W8[2] * ss * np.linalg.norm(q["virial"] - r["virial"]) * 1e-4 * np.linalg.norm(q["virial"])
        assert abs(loss[0] - loss_o) <= lb
        # parameters that no term reaches (a species pair absent from the cells) must be exactly zero
        zero = scale_o == 0.0
        assert np.all(g[zero] == 0.0)
        worst = np.max(np.abs(g[~zero] - grad_o[~zero]) / scale_o[~zero])
        assert worst <= 1e-4, worst


@pytest.fixture(scope="module", params=["stated", "smooth"])
def grad2048(request):
    pstar, p0, b, _ = make_grad_lev20.workload(request.param)
    cfgs = [b.config(k) for k in range(b.n_cfg)]
    refs, e_ref, f_ref, w_ref = _targets(oracle.Potential(pstar), cfgs)
    rng = np.random.default_rng(2048)
    pot = oracle.Potential(p0)
    dirs = []
    for _ in range(4):
        vxi, vc = rng.normal(size=p0.xi.shape), rng.normal(size=p0.c.shape)
        L0, dL = oloss.loss_and_directional(pot, cfgs, refs, W8, "vibrations", p0.xi, p0.c, vxi, vc)
        dirs.append((vxi, vc, L0, dL))
    return request.param, p0, b, e_ref, f_ref, w_ref, dirs


def test_config4_gradient_projections_all_2048_cells(gpu_lib, grad2048):
    recipe, p0, b, e_ref, f_ref, w_ref, dirs = grad2048
    assert b.n_cfg == 2048
    res = {}
    for precision in ("fp64", "fp32") if recipe == "smooth" else ("fp64",):
        model = mtp.Model.from_params(p0, precision)
        res[precision] = [t.cpu().numpy() for t in model.param_grad(*_batch_tensors(b), dev(e_ref), dev(f_ref),
                                                                       dev(w_ref), W8, "vibrations")]
    for vxi, vc, L0, dL in dirs:
        loss, dxi, dc = res["fp64"]
        assert loss[0] == pytest.approx(L0, rel=1e-10)
        got = float(dxi @ vxi + np.sum(dc * vc))
        size = float(np.abs(dxi) @ np.abs(vxi) + np.sum(np.abs(dc * vc)))
        assert abs(got - dL) <= 1e-8 * size
        if "fp32" not in res:
            continue
        # float path: the gradient vector within 1e-4 of its norm (normwise float bar), hence by
        # Cauchy-Schwarz a projection within 1e-4 |g| |v|; |g| from the double path, whose
        # projections match the oracle's above
        g64 = np.concatenate([dxi, dc.reshape(-1)])
        loss32, dxi32, dc32 = res["fp32"]
        got32 = float(dxi32 @ vxi + np.sum(dc32 * vc))
        vnorm = np.sqrt(vxi @ vxi + np.sum(vc * vc))
        assert abs(got32 - dL) <= 1e-4 * np.linalg.norm(g64) * vnorm


# ---------------------------------------------------------------------------------------------
# 1,048,576 atoms, lev_max 20, stated recipe
# ---------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def config5():
    cfg = synth.fcc_ternary()
    assert cfg.n == 1_048_576
    labels = synth.labels_from_level_table(levels.level_table(20))
    p = synth.scaled_params(20, 3, 8, 2.0, 5.0, labels, seed=5)
    which = np.sort(np.random.default_rng(55).choice(cfg.n, size=256, replace=False)).astype(np.int32)
    ref = oracle.Potential(p).eval_sampled(cfg, which)
    return cfg, p, which, ref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_config5_fcc64_ternary_lev20_sampled(gpu_lib, config5, precision):
    cfg, p, which, ref = config5
    model = mtp.Model.from_params(p, precision)
    out = model.eval(dev(cfg.pos), dev(cfg.types, torch.int32), dev(cfg.cell), site=True, b_atoms=True)
    idx = torch.as_tensor(which, dtype=torch.int64, device="cuda")
    site_all = out["site"]
    site = site_all[idx].cpu().numpy()
    B = out["b_atoms"][idx].cpu().numpy()
    F = out["forces"][idx].cpu().numpy()
    E = out["energy"].item()
    tol = TOL[precision]
    # site energies against the per-atom energy scale, basis rows against each column's scale
    assert np.abs(site - ref["site"]).max() <= tol["e"] * np.sqrt(np.mean(ref["site"] ** 2))
    colmax = np.abs(ref["b_atoms"]).max(0)
    assert np.all(np.abs(B - ref["b_atoms"]) <= tol["e"] * colmax + 1e-300)
    rms = np.sqrt(np.mean(ref["forces"] ** 2))
    assert np.sqrt(np.mean((F - ref["forces"]) ** 2)) <= tol["f"] * rms
    # properties of the whole cell: E is the sum of the site energies, the forces sum to zero
    s = site_all.sum().item()
    assert abs(E - s) <= 1e-12 * site_all.abs().sum().item()
    Fall = out["forces"]
    rms_all = Fall.pow(2).mean().sqrt().item()
    assert Fall.sum(0).abs().max().item() <= (1e-9 if precision == "fp64" else 1e-3) * rms_all * np.sqrt(cfg.n)
