"""The allocation-free MaxVol entry point agrees with the regular one.

mtp_select_active_set_noalloc serves callers that cannot allocate device memory; it keeps all of its
scratch in a fixed array inside the library.  Two calls in a row (on different matrices, so the
second starts from the first one's leftovers) must give the same rows and the same A^-1 as
mtp_select_active_set on the same input.  This file is collected last on purpose.
"""

import numpy as np
import pytest
import torch

from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu


def _matrix(K, m, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(K, m)) * 10.0 ** np.linspace(-3, 6, m)


def test_noalloc_matches_regular_entry_point_twice(gpu_lib):
    m = 17
    model = mtp.Model.from_params(synth.random_params(10, 1, 4, 2.0, 5.0, m, 0))
    for seed, K in ((11, 60), (12, 2 * m)):
        B = torch.as_tensor(_matrix(K, m, seed), dtype=torch.float64, device="cuda")
        sel_ref, swaps_ref, _ = model.select_active_set(B)
        _, ai_ref, _ = mtp.mtp_get_active_set(model.h, m)
        sel = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        ai = torch.zeros((m, m), dtype=torch.float64, device="cuda")
        swaps = mtp.mtp_select_active_set_noalloc(K, m, B, sel, ai)
        assert sel.cpu().tolist() == sel_ref.cpu().tolist()
        assert swaps == swaps_ref
        np.testing.assert_allclose(ai.cpu().numpy(), ai_ref, rtol=1e-10, atol=1e-10 * np.abs(ai_ref).max())


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu_lib):
    m = 100
    B = torch.zeros((6000, m), dtype=torch.float64, device="cuda")
    sel = torch.zeros(m, dtype=torch.int32, device="cuda")
    with pytest.raises(mtp.MTPError) as ei:
        mtp.mtp_select_active_set_noalloc(6000, m, B, sel)
    assert ei.value.code == 1
