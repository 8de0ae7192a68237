"""Bad inputs are refused with MTP_EINVAL, and a broken row reads as extrapolating.

* host-memory calls: a NaN or infinite position, a non-finite cell entry, a cell of zero volume and
  a species outside [0, S) are refused before anything is copied to the device;
* device-memory calls: the same positions and cells are reported by the neighbour build's own checks
  (its bin and wrap indices are clamped for any input, so nothing is read out of bounds), and the
  model evaluates normally afterwards (the error word is cleared);
* the extrapolation grade (Sec. 2.3) of a row with a NaN is +inf, not 0.
"""

import numpy as np
import pytest
import torch

from oracle import levels
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu


def _setup():
    b = synth.small_cells(n_cfg=3, n_lo=16, n_hi=40, seed=5)
    p = synth.random_params(8, 3, 4, 2.0, 5.0, len(levels.basis(8)), seed=2)
    return b, mtp.Model.from_params(p, "fp32")


def _bad_inputs(b):
    cases = []
    pos = b.pos.copy()
    pos[5, 1] = np.nan
    cases.append(("NaN position", pos, b.types, b.cells))
    pos = b.pos.copy()
    pos[0, 2] = np.inf
    cases.append(("infinite position", pos, b.types, b.cells))
    cells = b.cells.copy()
    cells[1, 2, 2] = np.nan
    cases.append(("NaN cell", b.pos, b.types, cells))
    cells = b.cells.copy()
    cells[2, 1] = cells[2, 0]  # two equal lattice vectors: zero volume
    cases.append(("singular cell", b.pos, b.types, cells))
    return cases


def _host_call(model, b, pos, types, cells):
    K, N = b.n_cfg, b.n_atoms
    e, f, w = np.zeros(K), np.zeros((N, 3)), np.zeros((K, 9))
    mtp.mtp_eval_batch(model.h, K, N, b.cfg_off, np.ascontiguousarray(pos), np.ascontiguousarray(types),
                       np.ascontiguousarray(cells.reshape(K, 9)), e, f, w, flags=mtp.HOST_MEMORY)
    return e


def test_host_memory_inputs_are_checked_before_copies(gpu_lib):
    b, model = _setup()
    launches = model.launch_count
    cases = _bad_inputs(b)
    types = b.types.copy()
    types[3] = 7
    cases.append(("species out of range", b.pos, types, b.cells))
    for what, pos, ty, cells in cases:
        with pytest.raises(mtp.MTPError) as ei:
            _host_call(model, b, pos, ty, cells)
        assert ei.value.code == 1, what
    assert model.launch_count == launches  # nothing reached the device
    e = _host_call(model, b, b.pos, b.types, b.cells)
    assert np.all(np.isfinite(e))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_device_memory_inputs_are_checked_by_the_neighbour_build(gpu_lib, precision):
    b, model = _setup()
    model = mtp.Model.from_params(synth.random_params(8, 3, 4, 2.0, 5.0, len(levels.basis(8)), seed=2), precision)
    off = torch.as_tensor(b.cfg_off, dtype=torch.int32, device="cuda")
    good = model.eval_batch(torch.as_tensor(b.pos, device="cuda"), torch.as_tensor(b.types, device="cuda"),
                            torch.as_tensor(b.cells, device="cuda"), off)["energy"].cpu().numpy()
    for what, pos, ty, cells in _bad_inputs(b):
        with pytest.raises(mtp.MTPError) as ei:
            model.eval_batch(torch.as_tensor(pos, device="cuda"), torch.as_tensor(ty, device="cuda"),
                             torch.as_tensor(cells, device="cuda"), off)
        assert ei.value.code == 1, what
        again = model.eval_batch(torch.as_tensor(b.pos, device="cuda"), torch.as_tensor(b.types, device="cuda"),
                                 torch.as_tensor(b.cells, device="cuda"), off)["energy"].cpu().numpy()
        np.testing.assert_allclose(again, good, rtol=1e-12)


def test_grade_of_a_nan_row_is_infinite(gpu_lib):
    m = 17
    model = mtp.Model.from_params(synth.random_params(10, 1, 4, 2.0, 5.0, m, 0))
    rng = np.random.default_rng(3)
    B = rng.normal(size=(40, m))
    model.select_active_set(torch.as_tensor(B, device="cuda"))
    rows = B[:4].copy()
    rows[1, 3] = np.nan
    rows[2, :] = np.nan
    g = model.grade(torch.as_tensor(rows, device="cuda")).cpu().numpy()
    assert np.isinf(g[1]) and np.isinf(g[2])
    assert np.isfinite(g[0]) and np.isfinite(g[3])
