"""Batched relaxation on the GPU (FIRE over positions and the cell, early stop on extrapolation)
against the oracle's relaxation (oracle/relax.py).

The potential is bounded below, as a relaxation needs: lev_max 6 with xi = (1, 0, 0, 0, 0), so that
E = sum_i M_{0,0}(n_i) is a pair potential 2 f_0(r), and the Chebyshev coefficients of f_0 fitted to
a Morse well (depth 0.3 eV, minimum at 2.6 Angstrom) times (R_cut - r)^2.  The other basis functions
carry no energy but enter the grades.

* six strained, noisy cells relax (positions and cell) to the oracle's minima: same outcome,
  energies within 1e-9 relative, positions and cells within 1e-5 Angstrom (both runs stop within the
  force tolerance of the same minimum), forces below the tolerance;
* a relaxation started far from the active set's configurations stops at the same step as the
  oracle when its grade reaches gamma_break, with the same coordinates.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import levels, maxvol, relax
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu

RMIN, RCUT = 1.5, 5.0


def morse_params():
    L, NQ = 6, 8
    m = len(levels.basis(L))
    r = np.linspace(1.8, 4.95, 400)
    x = (2 * r - RMIN - RCUT) / (RCUT - RMIN)
    eps, alpha, r0 = 0.3, 1.5, 2.6
    h = eps / (RCUT - r0) ** 2 * (np.exp(-2 * alpha * (r - r0)) - 2 * np.exp(-alpha * (r - r0)))
    T = np.polynomial.chebyshev.chebvander(x, NQ - 1)
    coef = np.linalg.lstsq(T, h, rcond=None)[0]
    c = np.zeros((1, 1, (L - 2) // 4 + 1, NQ))
    c[0, 0, 0] = coef
    c[0, 0, 1] = 0.05 * np.random.default_rng(5).normal(size=NQ)  # f_1 enters only the grades
    xi = np.zeros(m)
    xi[0] = 1.0
    return synth.Params(L, 1, NQ, RMIN, RCUT, xi, c)


def cells(n_cfg, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_cfg):
        kind = ["fcc", "hcp"][k % 2]
        cfg = synth.perturbed(kind, (2, 2, 2), 0.06, rng)
        e = rng.uniform(-0.03, 0.03, size=(3, 3))
        strain = np.eye(3) + 0.5 * (e + e.T)
        out.append(synth.Config(cfg.pos @ strain.T, cfg.types, cfg.cell @ strain.T))
    return out


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def oracle_relax(pot, cfg, **kw):
    def evaluate(x, H):
        r = pot.eval(synth.Config(x, cfg.types, H))
        return r["energy"], r["forces"], r["virial"]
    return relax.relax(evaluate, cfg.pos, cfg.cell, **kw)


def test_batch_relaxes_to_oracle_minima(gpu_lib):
    p = morse_params()
    pot = oracle.Potential(p)
    cfgs = cells(6, 11)
    kw = dict(fmax=1e-4, smax=1e-5, dt=0.05, dt_max=0.5, max_steps=3000)
    refs = [oracle_relax(pot, c, **kw) for c in cfgs]
    assert all(r["converged"] for r in refs)
    b = synth.pack(cfgs)
    model = mtp.Model.from_params(p, "fp64")
    pos, cl = dev(b.pos), dev(b.cells)
    energy, steps, status = model.relax_batch(pos, dev(b.types, torch.int32), cl, dev(b.cfg_off, torch.int32), **kw)
    assert status.tolist() == [1] * len(cfgs)
    e = energy.cpu().numpy()
    P, C = pos.cpu().numpy(), cl.cpu().numpy()
    for k, (c, r) in enumerate(zip(cfgs, refs)):
        a0, a1 = b.cfg_off[k], b.cfg_off[k + 1]
        assert e[k] == pytest.approx(r["energy"], rel=1e-9)
        np.testing.assert_allclose(P[a0:a1], r["pos"], atol=1e-5)
        np.testing.assert_allclose(C[k], r["cell"], atol=1e-5)
        # the device's final state is a minimum: forces and stress below the tolerances
        fin = pot.eval(synth.Config(P[a0:a1], c.types, C[k]))
        assert np.abs(fin["forces"]).max() <= 1e-4
        assert np.abs(fin["virial"]).max() / abs(np.linalg.det(C[k])) <= 1e-5
        assert abs(int(steps[k]) - r["steps"]) <= max(3, r["steps"] // 20), (steps[k], r["steps"])


def gamma_case():
    """A start (strained, noisy), an active set from small perturbations of it, and gamma_break placed
    (at least 2% away from every grade) where the oracle's run first exceeds it."""
    p = morse_params()
    pot = oracle.Potential(p)
    m = len(p.xi)
    rng = np.random.default_rng(21)
    start = cells(1, 22)[0]
    pool = [synth.Config(start.pos + rng.normal(0, 0.02, size=start.pos.shape), start.types, start.cell)
            for _ in range(3 * m)]
    B = np.array([pot.eval(c, want_b=True)["b_atoms"].sum(0) for c in pool])
    sel, _, _ = maxvol.maxvol(B)
    A = B[sel]

    def grade(x, H):
        return maxvol.grades(pot.eval(synth.Config(x, start.types, H), want_b=True)["b_atoms"].sum(0)[None], A)[0]

    kw = dict(fmax=1e-4, smax=1e-5, dt=0.05, dt_max=0.5, max_steps=400)
    g = np.array(oracle_relax(pot, start, grade=grade, **kw)["gammas"])
    k = next(k for k in range(3, len(g)) if g[k] > 1.05 * g[:k].max() and g[k] > 1.5)
    gb = float(np.sqrt(g[:k].max() * g[k]))
    ref = oracle_relax(pot, start, grade=grade, gamma_break=gb, **kw)
    return p, start, B, gb, kw, ref, k


def test_relaxation_stops_at_gamma_break(gpu_lib):
    p, start, B, gb, kw, ref, k = gamma_case()
    assert ref["stopped"] and ref["steps"] == k
    model = mtp.Model.from_params(p, "fp64")
    model.select_active_set(dev(B))
    b = synth.pack([start])
    pos, cl = dev(b.pos), dev(b.cells)
    energy, steps, status = model.relax_batch(pos, dev(b.types, torch.int32), cl, dev(b.cfg_off, torch.int32),
                                              gamma_break=gb, **kw)
    assert status.tolist() == [2] and steps.tolist() == [k]
    np.testing.assert_allclose(pos.cpu().numpy(), ref["pos"], atol=1e-9)
    np.testing.assert_allclose(cl.cpu().numpy()[0], ref["cell"], atol=1e-9)
