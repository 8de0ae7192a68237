"""Model files on the GPU: a model written by mtp_save and read by mtp_load evaluates and grades
exactly like the original (same parameters, settings and active set), and saving the loaded model
writes the same file."""

import numpy as np
import pytest
import torch

from paper_2007_08555_gb300 import codegen, mtp, synth

pytestmark = pytest.mark.gpu


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_save_load_round_trip(gpu_lib, tmp_path, precision):
    L, S = 12, 2
    b = synth.small_cells(n_cfg=6, n_lo=16, n_hi=64, seed=21)
    p = synth.random_params(L, S, 6, 2.0, 5.0, codegen.build_basis(L).m, seed=5)
    model = mtp.Model.from_params(p, precision)
    model.set_neighbor_capacity(160)
    model.set_threads_per_atom(2, 4)
    m = model.m
    rng = np.random.default_rng(3)
    A = rng.normal(size=(m, m)) + 4.0 * np.eye(m)
    mtp.mtp_set_active_set(model.h, A)

    path = tmp_path / "pot.txt"
    model.save(str(path))
    loaded = mtp.Model.load(str(path))
    assert loaded.m == m and loaded.n_species == S and loaded.n_radial == 6
    assert loaded.precision == model.precision
    assert loaded.level_table().tolist() == model.level_table().tolist()

    A0, Ai0, r0 = mtp.mtp_get_active_set(model.h, m)
    A1, Ai1, r1 = mtp.mtp_get_active_set(loaded.h, m)
    assert np.array_equal(A0, A1) and np.array_equal(Ai0, Ai1) and np.array_equal(r0, r1)

    pos, types, cells, off = (dev(b.pos, torch.float64), dev(b.types % S, torch.int32),
                              dev(b.cells, torch.float64), dev(b.cfg_off, torch.int32))
    o0 = model.eval_batch(pos, types, cells, off, b_rows=True, grade_cfg=True)
    o1 = loaded.eval_batch(pos, types, cells, off, b_rows=True, grade_cfg=True)
    # forces come from a deterministic gather; the per-configuration sums use double atomics
    assert torch.equal(o0["forces"], o1["forces"])
    np.testing.assert_allclose(o1["energy"].cpu().numpy(), o0["energy"].cpu().numpy(), rtol=1e-13, atol=0)
    np.testing.assert_allclose(o1["virial"].cpu().numpy(), o0["virial"].cpu().numpy(), rtol=1e-12,
                               atol=1e-12 * float(o0["virial"].abs().max()))
    rows = o0["b_rows"].contiguous()
    assert torch.equal(model.grade(rows), loaded.grade(rows))

    again = tmp_path / "again.txt"
    loaded.save(str(again))
    assert again.read_text() == path.read_text()


def test_model_without_active_set(gpu_lib, tmp_path):
    p = synth.random_params(8, 1, 4, 2.0, 5.0, codegen.build_basis(8).m, seed=1)
    model = mtp.Model.from_params(p, "fp64")
    model.set_skin(0.3)
    path = tmp_path / "pot.txt"
    model.save(str(path))
    assert "active_set 0" in path.read_text() and "skin 0.29999999999999999" in path.read_text()
    loaded = mtp.Model.load(str(path))
    with pytest.raises(mtp.MTPError) as ei:
        mtp.mtp_get_active_set(loaded.h, loaded.m)
    assert ei.value.code == 7
