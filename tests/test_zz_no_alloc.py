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


def _scratch_doubles(n, m):
    """Doubles of the fixed scratch array used for n rows of m columns (the layout stated in mtp.h)."""
    nm, mm = n * m, m * m
    return 2 * nm + max(nm, 2 * mm) + 2 * mm + 3 * m + n + (n + m + 3) // 2 + 1


def test_noalloc_accepts_the_largest_size_that_fits_and_rejects_one_more_row(gpu_lib):
    m = 116
    n = m
    while _scratch_doubles(n + 1, m) <= 1 << 19:
        n += 1
    assert n == 1421  # the figure stated in mtp.h
    model = mtp.Model.from_params(synth.random_params(16, 1, 4, 2.0, 5.0, m, 0))
    B = torch.as_tensor(_matrix(n + 1, m, 21), dtype=torch.float64, device="cuda")
    sel = torch.full((m,), -1, dtype=torch.int32, device="cuda")
    swaps = mtp.mtp_select_active_set_noalloc(n, m, B[:n].contiguous(), sel)
    sel_ref, swaps_ref, _ = model.select_active_set(B[:n].contiguous())
    assert sel.cpu().tolist() == sel_ref.cpu().tolist() and swaps == swaps_ref
    with pytest.raises(mtp.MTPError) as ei:
        mtp.mtp_select_active_set_noalloc(n + 1, m, B, sel)
    assert ei.value.code == 1
