"""Runs the float evaluation (neighbour build + E/F/W) of one periodic cell alone, for kernel
profiling and timing at sizes between the 16k-atom and the 1M-atom workloads.

Usage: python -m paper_2007_08555_gb300.profile_eval [reps_per_side] [lev_max] [repeats] [lanes_moments]
       [lanes_pairs] [cell]
cell "ternary" (the default): fcc with a = 3.6 A, reps^3 conventional cells (4 reps^3 atoms), three
species at random, no displacements; parameters on the stated recipe (R_min 2 A, c ~ N(0, 0.1), xi
scaled per basis function, seed 5).
cell "binary": the headline cell, fcc reps^3 with two species at random 50/50 occupancy and sigma =
0.15 A displacements, parameters xi ~ N(0, 1e-2), c ~ N(0, 0.1) (seed 2), as timed by bench.py.
Lanes per atom of the pair kernels as given, autotuned when 0 (the default).  The first evaluation is
eager, the second is captured into a CUDA graph, later ones replay it.  Prints the CUDA-event time per
evaluation and its phases.
"""

import sys

import numpy as np
import torch

from . import codegen, mtp, synth


def main():
    reps = int(sys.argv[1]) if len(sys.argv) > 1 else 32
    L = int(sys.argv[2]) if len(sys.argv) > 2 else 20
    repeats = int(sys.argv[3]) if len(sys.argv) > 3 else 5
    lanes = (int(sys.argv[4]) if len(sys.argv) > 4 else 0, int(sys.argv[5]) if len(sys.argv) > 5 else 0)
    kind = sys.argv[6] if len(sys.argv) > 6 else "ternary"
    if kind == "binary":
        cfg = synth.fcc_binary(reps=reps, seed=2)
        p = synth.random_params(L, 2, 8, 2.0, 5.0, codegen.build_basis(L).m, seed=2)
    elif kind == "ternary":
        cfg = synth.fcc_ternary(reps=reps)
        labels = synth.labels_from_level_table(codegen.level_table(codegen.build_basis(L)))
        p = synth.scaled_params(L, 3, 8, 2.0, 5.0, labels, seed=5)
    else:
        raise SystemExit(f"unknown cell {kind!r} (binary or ternary)")
    d = lambda a, t=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    pos, types = d(cfg.pos), d(cfg.types, torch.int32)
    cells, off = d(cfg.cell.reshape(1, 3, 3)), d(np.array([0, cfg.n]), torch.int32)
    model = mtp.Model.from_params(p, "fp32")
    if lanes[0] and lanes[1]:
        model.set_threads_per_atom(*lanes)
        tuned = lanes
    else:
        tuned = model.autotune(pos, types, cells, off)[:2]  # lanes per atom of the pair kernels
    out = model.eval_batch(pos, types, cells, off)
    torch.cuda.synchronize()
    mtp.mtp_profile(model.h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(repeats):
        out = model.eval_batch(pos, types, cells, off, out=out)
    e1.record()
    torch.cuda.synchronize()
    phases, calls = mtp.mtp_profile_read(model.h)
    ms = e0.elapsed_time(e1) / repeats
    print(f"fcc {reps}^3 {kind}, {cfg.n} atoms, lev_max {L}, lanes per atom {tuned}: {ms:.4f} ms per "
          "evaluation; phases (ms) "
          + ", ".join(f"{k} {v / max(calls, 1):.4f}" for k, v in phases.items()))


if __name__ == "__main__":
    main()
