"""Runs the tensor-core grade (MTP_FP32_TC) alone on synthetic rows, for kernel profiling and timing.

Usage: python -m paper_2007_08555_gb300.profile_grade_tc [n_rows] [lev_max] [repeats]
Rows are random with columns spanning nine decades (as in the tests); the active set is chosen by
MaxVol over the first 2 m rows.  Prints the CUDA-event time per grade call of the tensor-core and
the double-precision products.
"""

import sys

import numpy as np
import torch

from . import codegen, mtp, synth


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 303_192
    L = int(sys.argv[2]) if len(sys.argv) > 2 else 16
    reps = int(sys.argv[3]) if len(sys.argv) > 3 else 10
    m = codegen.build_basis(L).m
    rng = np.random.default_rng(1)
    B = torch.as_tensor(rng.normal(size=(n, m)) * 10.0 ** np.linspace(-3, 6, m), device="cuda")
    p = synth.random_params(L, 1, 4, 2.0, 5.0, m, 0)
    out = {}
    for prec in ("fp32_tc", "fp64"):
        model = mtp.Model.from_params(p, prec)
        model.select_active_set(B[:2 * m].contiguous())
        g = torch.empty(n, dtype=torch.float64, device="cuda")
        mtp.mtp_grade(model.h, n, B, g)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            mtp.mtp_grade(model.h, n, B, g, flags=mtp.ASYNC)
        e1.record()
        torch.cuda.synchronize()
        out[prec] = (e0.elapsed_time(e1) / reps, g.clone())
    rel = float(((out["fp32_tc"][1] - out["fp64"][1]).abs() / out["fp64"][1]).max())
    print(f"n {n} m {m}: tensor cores {out['fp32_tc'][0]:.4f} ms, double product {out['fp64'][0]:.4f} ms, "
          f"max rel diff {rel:.2e}")


if __name__ == "__main__":
    main()
