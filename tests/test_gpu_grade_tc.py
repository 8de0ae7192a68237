"""The extrapolation grade (Sec. 2.3) on the tensor cores (MTP_FP32_TC) against the double-precision
product and the oracle.

The tensor-core product is exact on 56-bit roundings of b D and (A D)^-1 apart from the dropped
digit pairs, so against the double-precision grade of the same rows and the same A^-1 it is held to
  |gamma_tc - gamma_64| <= 2^-24 gamma_64 + 1e-14 2^E_r max_j 2^F_j + 1e-15 max_j (|b_r| |A^-1|)_j
(the final rounding to float, correctly rounded; the rounding of the operands and the dropped pairs, below ~1.5e-14 of
the row and column scales 2^E_r <= 4 max_k |b_rk D_k|, 2^F_j <= 4 max_k |G_kj| in the worst case at
m = 460; the double-precision product's own error).  Matrices up to m = 460 (lev_max 20) with columns spanning nine decades,
real basis rows of small cells (grades per configuration and per atom), and a row with NaN.
"""

import numpy as np
import pytest
import torch

from oracle import levels, maxvol
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def tc_bound(B, A, Ai, g64):
    """The bound of the module docstring, from the rows B, the active set A and the device's A^-1."""
    d = 2.0 ** -np.ceil(np.log2(np.abs(A).max(0) * (1 + 1e-15)))
    Bs = np.abs(B) * d
    G = np.abs(Ai) / d[:, None]
    row = 4.0 * Bs.max(1)  # 2^E_r <= 4 max_k |b_rk D_k|
    col = 4.0 * G.max(0)
    return 2.0 ** -24 * (1 + 1e-12) * g64 + 2e-14 * row * col.max() + 1e-15 * (np.abs(B) @ np.abs(Ai)).max(1)


@pytest.mark.parametrize("K,m,L,seed", [(40, 9, 8, 1), (60, 17, 10, 3), (232, 116, 16, 2), (700, 460, 20, 4)])
def test_tc_grade_matches_double_product_and_oracle(gpu_lib, K, m, L, seed):
    p = synth.random_params(L, 1, 4, 2.0, 5.0, m, 0)
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(K, m)) * 10.0 ** np.linspace(-3, 6, m)
    m64 = mtp.Model.from_params(p, "fp64")
    mtc = mtp.Model.from_params(p, "fp32_tc")
    sel64, _, _ = m64.select_active_set(dev(B))
    sel, _, _ = mtc.select_active_set(dev(B))
    assert sel.cpu().tolist() == sel64.cpu().tolist()
    _, Ai, _ = mtp.mtp_get_active_set(mtc.h, m)
    g64 = m64.grade(dev(B)).cpu().numpy()
    gtc = mtc.grade(dev(B)).cpu().numpy()
    A = B[sel.cpu().numpy()]
    bound = tc_bound(B, A, Ai, g64)
    assert np.all(np.abs(gtc - g64) <= bound), float(np.max(np.abs(gtc - g64) / bound))
    np.testing.assert_allclose(gtc[sel.cpu().numpy()], 1.0, rtol=1e-6)
    g_ref = maxvol.grades(B, A)
    np.testing.assert_allclose(gtc, g_ref, rtol=1e-9 + 2.0 ** -23)


@pytest.mark.parametrize("L", [10, 16])
def test_tc_grades_per_configuration_and_atom(gpu_lib, L):
    m = len(levels.basis(L))
    p = synth.random_params(L, 3, 8, 2.0, 5.0, m, seed=70 + L)
    b = synth.small_cells(n_cfg=2 * m + 40, n_lo=8, n_hi=64, seed=71 + L)
    pos, types, cells, off = dev(b.pos), dev(b.types, torch.int32), dev(b.cells), dev(b.cfg_off, torch.int32)
    m64 = mtp.Model.from_params(p, "fp64")
    rows = m64.eval_batch(pos, types, cells, off, b_rows=True)["b_rows"]
    m32 = mtp.Model.from_params(p, "fp32")
    mtc = mtp.Model.from_params(p, "fp32_tc")
    for mod in (m32, mtc):
        mod.select_active_set(rows[:2 * m].contiguous())
    A, Ai, _ = mtp.mtp_get_active_set(mtc.h, m)
    A32, Ai32, _ = mtp.mtp_get_active_set(m32.h, m)
    np.testing.assert_array_equal(Ai, Ai32)
    o32 = m32.eval_batch(pos, types, cells, off, b_rows=True, b_atoms=True, grade_cfg=True, grade_atom=True)
    otc = mtc.eval_batch(pos, types, cells, off, b_rows=True, b_atoms=True, grade_cfg=True, grade_atom=True)
    for key, rk in (("grade_cfg", "b_rows"), ("grade_atom", "b_atoms")):
        Bn = otc[rk].cpu().numpy()
        np.testing.assert_array_equal(Bn, o32[rk].cpu().numpy())  # same float evaluation
        g64 = o32[key].cpu().numpy()
        gtc = otc[key].cpu().numpy()
        bound = tc_bound(Bn, A, Ai, g64)
        assert np.all(np.abs(gtc - g64) <= bound), (key, float(np.max(np.abs(gtc - g64) / bound)))
    # repeated identical calls replay the captured graph with the tensor-core kernel inside
    first = {k: otc[k].cpu().numpy().copy() for k in ("grade_cfg", "grade_atom")}
    for _ in range(2):
        otc = mtc.eval_batch(pos, types, cells, off, out=otc)
    for k in first:
        np.testing.assert_array_equal(otc[k].cpu().numpy(), first[k])


def test_tc_grade_of_nan_row_is_infinite(gpu_lib):
    m = 17
    mtc = mtp.Model.from_params(synth.random_params(10, 1, 4, 2.0, 5.0, m, 0), "fp32_tc")
    rng = np.random.default_rng(3)
    B = rng.normal(size=(40, m))
    mtc.select_active_set(dev(B))
    rows = B[:4].copy()
    rows[1, 3] = np.nan
    rows[2, 5] = np.inf
    g = mtc.grade(dev(rows)).cpu().numpy()
    assert np.isinf(g[1]) and np.isinf(g[2]) and np.isfinite(g[0]) and np.isfinite(g[3])
    assert np.all(g[[0, 3]] <= 1.0 + 1e-3 + 1e-6)  # rows of the pool: dominated by the active set
