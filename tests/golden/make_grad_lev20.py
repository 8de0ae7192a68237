"""Writes grad_lev20_<recipe>_cells.txt: the oracle's training-loss gradient (Sec. 2.2, Eq. 12) for
four cells of the lev_max-20 training workload, read by tests/test_gpu_full_size.py and
tests/test_gpu_autograd.py.

Calls only the oracle (oracle/) and the seeded input generators.  Inputs: the 2048 training cells
of 32-128 atoms (seed 4), 3 species, lev_max 20, N_Q 8, R_cut 5, xi scaled per basis function;
recipe "stated": R_min 2, c ~ N(0, 0.1); recipe "smooth": R_min 1, c ~ N(0, 0.1) damped by 0.5^b
(the recipe whose gradient stays within float range; the stated one reaches 1e57 on the 2048
cells); targets E, F, W at the hidden parameters (seed 40), gradient at seed 41, weights
1 / 0.01 / 0.001, "vibrations" scaling.  The four cells are the four smallest of the first 64
(stable order).  Besides the gradient, every entry a gets the componentwise scale
    sum_k [ 2 s_e w_e |dE_k| |dE_k/da| + 2 s_f w_f sum_i,c |dF_ikc| |dF_ikc/da|
            + 2 s_s w_s sum_bc |dW_kbc| |dW_kbc/da| ]
(d = model - target), the size of the terms the entry sums, against which a float evaluation's
error is judged.

Run: python tests/golden/make_grad_lev20.py stated|smooth   (a few minutes on 8 cores)
"""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import levels, loss as oloss  # noqa: E402
from paper_2007_08555_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = (1.0, 0.01, 0.001)
RECIPES = {"stated": dict(r_min=2.0, radial_decay=1.0), "smooth": dict(r_min=1.0, radial_decay=0.5)}


def out_path(recipe):
    return os.path.join(HERE, f"grad_lev20_{recipe}_cells.txt")


def workload(recipe="stated"):
    labels = synth.labels_from_level_table(levels.level_table(20))
    r = RECIPES[recipe]
    pstar = synth.scaled_params(20, 3, 8, r["r_min"], 5.0, labels, seed=40, radial_decay=r["radial_decay"])
    p0 = synth.scaled_params(20, 3, 8, r["r_min"], 5.0, labels, seed=41, radial_decay=r["radial_decay"])
    b = synth.training_cells(n_cfg=2048, seed=4)
    n = np.diff(b.cfg_off)
    cells = np.sort(np.argsort(n[:64], kind="stable")[:4])
    return pstar, p0, b, cells


def main(recipe):
    pstar, p0, b, cells = workload(recipe)
    cfgs = [b.config(int(k)) for k in cells]
    refs = [oracle.Potential(pstar).eval(c) for c in cfgs]
    pot = oracle.Potential(p0)
    we, wf, ws = WEIGHTS
    nx, nc = p0.xi.size, p0.c.size
    grad = np.zeros(nx + nc)
    scale = np.zeros(nx + nc)
    loss = 0.0
    for a in range(nx + nc):
        v = np.zeros(nx + nc)
        v[a] = 1.0
        vxi, vc = v[:nx], v[nx:].reshape(p0.c.shape)
        for cfg, ref in zip(cfgs, refs):
            r = pot.eval(cfg, dxi=vxi, dc=vc)
            se, sf, ss = oloss.scale("vibrations", cfg.n)
            de = r["energy"] - ref["energy"]
            dfo = r["forces"] - ref["forces"]
            dw = r["virial"] - ref["virial"]
            grad[a] += (2 * se * we * de * r["d_energy"] + 2 * sf * wf * np.sum(dfo * r["d_forces"])
                        + 2 * ss * ws * np.sum(dw * r["d_virial"]))
            scale[a] += (2 * se * we * abs(de * r["d_energy"]) + 2 * sf * wf * np.sum(np.abs(dfo * r["d_forces"]))
                         + 2 * ss * ws * np.sum(np.abs(dw * r["d_virial"])))
            if a == 0:
                loss += se * we * de ** 2 + sf * wf * np.sum(dfo ** 2) + ss * ws * np.sum(dw ** 2)
    with open(out_path(recipe), "w") as f:
        f.write(f"# oracle gradient of the Eq. 12 loss, lev_max 20, recipe {recipe}; written by make_grad_lev20.py\n")
        f.write("cells " + " ".join(str(int(k)) for k in cells) + "\n")
        f.write(f"loss {loss:.17e}\n")
        for a in range(nx + nc):
            f.write(f"{grad[a]:.17e} {scale[a]:.17e}\n")


def read(recipe="stated"):
    """(cells, loss, gradient [820], scale [820]) from the stored file."""
    with open(out_path(recipe)) as f:
        lines = [l for l in f if not l.startswith("#")]
    cells = np.array([int(x) for x in lines[0].split()[1:]])
    loss = float(lines[1].split()[1])
    vals = np.array([[float(x) for x in l.split()] for l in lines[2:]])
    return cells, loss, vals[:, 0], vals[:, 1]


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "stated")
