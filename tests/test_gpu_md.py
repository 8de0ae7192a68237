"""GPU parity of the MD step: neighbour lists with a skin and velocity Verlet.

* an evaluation that refreshes r_ij from a list built with a skin equals a fresh evaluation and the
  oracle at the displaced positions;
* the device trajectory (FP64 path, rebuilds forced by a small skin) equals a numpy velocity Verlet
  driven by the oracle's forces;
* the FP32 path conserves the total energy over 100 steps of 1 fs.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import levels
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu

MASSES = [26.98, 58.69, 63.55]
MVV = 103.642696


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def scaled(L, S, seed, decay=1.0, r_min=2.0):
    return synth.scaled_params(L, S, 8, r_min, 5.0, synth.labels_from_level_table(levels.level_table(L)), seed,
                               radial_decay=decay)


@pytest.mark.parametrize("precision,tol_e,tol_f", [("fp64", 1e-10, 1e-10), ("fp32", 1e-5, 1e-4)])
def test_refresh_matches_fresh_build(gpu_lib, precision, tol_e, tol_f):
    rng = np.random.default_rng(3)
    cfg = synth.perturbed("fcc", (4, 4, 4), 0.08, rng, n_species=2)
    p = scaled(12, 2, 4)
    model = mtp.Model.from_params(p, precision)
    model.set_skin(0.5)
    types, cell = dev(cfg.types, torch.int32), dev(cfg.cell)
    model.eval(dev(cfg.pos), types, cell)  # builds the list with the skin
    moved = cfg.pos + rng.uniform(-0.12, 0.12, size=cfg.pos.shape)
    out = model.eval(dev(moved), types, cell, flags=mtp.REUSE_NEIGHBORS)
    fresh = mtp.Model.from_params(p, precision).eval(dev(moved), types, cell)
    ref = oracle.Potential(p).eval(synth.Config(moved, cfg.types, cfg.cell))
    for o in (out, fresh):
        assert abs(o["energy"].item() - ref["energy"]) <= tol_e * abs(ref["energy"])
        F = o["forces"].cpu().numpy()
        assert np.sqrt(np.mean((F - ref["forces"]) ** 2)) <= tol_f * np.sqrt(np.mean(ref["forces"] ** 2))
    np.testing.assert_allclose(out["virial"].cpu().numpy(), ref["virial"], rtol=10 * tol_f,
                               atol=tol_f * np.abs(ref["virial"]).max())


def test_verlet_matches_oracle_driven_verlet(gpu_lib):
    rng = np.random.default_rng(11)
    cfg = synth.perturbed("fcc", (3, 3, 3), 0.05, rng, n_species=3)
    p = scaled(10, 3, 12)
    v0 = synth.maxwell_velocities(cfg.types, MASSES, 300.0, seed=12)
    dt, steps = 1.0, 12
    model = mtp.Model.from_params(p, "fp64")
    model.set_skin(0.04)  # small: forces several rebuilds within the run
    x = dev(cfg.pos)
    v = dev(v0)
    ep, ek, rebuilds = model.md_run(x, v, dev(cfg.types, torch.int32), dev(cfg.cell), MASSES, dt, steps)
    assert rebuilds >= 2
    # the same integrator in numpy with the oracle's forces
    pot = oracle.Potential(p)
    m = np.array(MASSES)[cfg.types][:, None] * MVV
    xs, vs = cfg.pos.copy(), v0.copy()
    r = pot.eval(synth.Config(xs, cfg.types, cfg.cell))
    e_ref = [r["energy"]]
    F = r["forces"]
    for _ in range(steps):
        vs = vs + 0.5 * dt * F / m
        xs = xs + dt * vs
        r = pot.eval(synth.Config(xs, cfg.types, cfg.cell))
        F = r["forces"]
        vs = vs + 0.5 * dt * F / m
        e_ref.append(r["energy"])
    np.testing.assert_allclose(x.cpu().numpy(), xs, rtol=0, atol=1e-9)
    np.testing.assert_allclose(v.cpu().numpy(), vs, rtol=0, atol=1e-11)
    np.testing.assert_allclose(ep, e_ref, rtol=1e-9, atol=1e-9 * np.abs(e_ref).max())
    np.testing.assert_allclose(ek[-1], 0.5 * np.sum(m * vs ** 2), rtol=1e-10)


def test_fp32_energy_conservation(gpu_lib):
    # smooth radial functions (damped Chebyshev coefficients): a well-resolved trajectory
    rng = np.random.default_rng(21)
    cfg = synth.perturbed("fcc", (6, 6, 6), 0.0, rng, n_species=3)
    p = scaled(16, 3, 22, decay=0.5, r_min=1.0)
    v0 = synth.maxwell_velocities(cfg.types, MASSES, 300.0, seed=23)
    runs = {}
    for prec in ("fp32", "fp64"):
        model = mtp.Model.from_params(p, prec)
        model.set_skin(0.5)
        x, v = dev(cfg.pos), dev(v0)
        ep, ek, rebuilds = model.md_run(x, v, dev(cfg.types, torch.int32), dev(cfg.cell), MASSES, 1.0, 100)
        runs[prec] = (ep + ek) / cfg.n
    for prec, et in runs.items():
        assert np.isfinite(et).all()
        assert np.abs(et - et[0]).max() <= 1e-5, (prec, np.abs(et - et[0]).max())
    # the float trajectory follows the double one
    assert np.abs(runs["fp32"] - runs["fp64"]).max() <= 1e-5
