"""The autotuner of the batched launch and the packed-atom work queue.

* mtp_autotune times all 16 lanes-per-atom choices on a batch of small cells and records the fastest
  for the batch's size class; a model left on automatic choice then evaluates with that choice,
  and its results equal the oracle's at the bars and the explicitly configured model's to rounding;
* the work queues of the moment and pair-gradient kernels start from zero at every evaluation:
  repeated evaluations (graph replays), a refresh with a skin and a loss gradient all agree.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import levels
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_autotune_records_and_uses_the_fastest_choice(gpu_lib):
    L = 12
    b = synth.small_cells(n_cfg=40, n_lo=8, n_hi=128, seed=91)
    p = synth.random_params(L, 3, 8, 2.0, 5.0, len(levels.basis(L)), seed=92)
    pos, types, cells, off = dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32)
    model = mtp.Model.from_params(p, "fp32")
    bm, bp, times = model.autotune(pos, types, cells, off)
    assert bm in (1, 2, 4, 8) and bp in (1, 2, 4, 8)
    assert np.all(times > 0) and times[int(np.log2(bm)), int(np.log2(bp))] == times.min()
    auto = model.eval_batch(pos, types, cells, off)
    fixed = mtp.Model.from_params(p, "fp32")
    fixed.set_threads_per_atom(bm, bp)
    ref = fixed.eval_batch(pos, types, cells, off)
    np.testing.assert_allclose(auto["forces"].cpu().numpy(), ref["forces"].cpu().numpy(), rtol=0, atol=0)
    np.testing.assert_allclose(auto["energy"].cpu().numpy(), ref["energy"].cpu().numpy(), rtol=1e-13)
    pot = oracle.Potential(p)
    e = auto["energy"].cpu().numpy()
    for k in range(b.n_cfg):
        r = pot.eval(b.config(k))
        assert abs(e[k] - r["energy"]) <= 1e-5 * max(abs(r["energy"]), 1e-12), k


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_work_queues_restart_every_evaluation(gpu_lib, precision):
    L = 10
    b = synth.small_cells(n_cfg=12, n_lo=16, n_hi=96, seed=93)
    p = synth.random_params(L, 3, 8, 2.0, 5.0, len(levels.basis(L)), seed=94)
    pos, types, cells, off = dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32)
    model = mtp.Model.from_params(p, precision)
    first = model.eval_batch(pos, types, cells, off)
    out = None
    for _ in range(4):  # eager, captured, replays
        out = model.eval_batch(pos, types, cells, off, out=out)
        np.testing.assert_allclose(out["forces"].cpu().numpy(), first["forces"].cpu().numpy(), rtol=1e-12,
                                   atol=1e-12 * np.abs(first["forces"].cpu().numpy()).max())
    # a loss gradient in between, then a refresh of r_ij with a skin (no rebuild): same results
    e_ref = first["energy"] * 1.01
    model.param_grad(pos, types, cells, off, e_ref, first["forces"], first["virial"].reshape(-1, 9).contiguous())
    model.set_skin(0.3)
    model.eval_batch(pos, types, cells, off)
    again = model.eval_batch(pos, types, cells, off, flags=mtp.REUSE_NEIGHBORS)
    # the list with a skin holds more pairs, which changes how pairs fall on the lanes of an atom, so
    # the float path agrees to rounding of its sums only
    np.testing.assert_allclose(again["energy"].cpu().numpy(), first["energy"].cpu().numpy(),
                               rtol=1e-12 if precision == "fp64" else 1e-4)
