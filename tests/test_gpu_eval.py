"""GPU parity of the evaluation path (through the C ABI) against the FP64 oracle.

Bars: neighbour lists and level tables bit-exact; FP64 path within 1e-10 (relative, per the
spec tolerance of the double-precision path); FP32 path within 1e-5 relative in the
energy (per atom and per configuration), 1e-4 relative to the RMS force, 1e-4 relative in the
virial (Frobenius norm).
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import levels, maxvol
from paper_2007_08555_gb300 import mtp, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(e=1e-10, f=1e-10, w=1e-10), "fp32": dict(e=1e-5, f=1e-4, w=1e-4)}


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def batch_tensors(b):
    return (dev(b.pos, torch.float64), dev(b.types, torch.int32), dev(b.cells, torch.float64),
            dev(b.cfg_off, torch.int32))


def params(L, S, seed, NQ=8):
    return synth.random_params(L, S, NQ, 2.0, 5.0, len(levels.basis(L)), seed)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def check_config(out_e, out_f, out_w, ref, n, tol, msg=""):
    assert abs(out_e - ref["energy"]) / n <= tol["e"] * max(abs(ref["energy"]) / n, 1e-12), msg
    F = ref["forces"]
    rms = np.sqrt(np.mean(F ** 2)) if F.size else 1.0
    if F.size:
        assert np.sqrt(np.mean((out_f - F) ** 2)) <= tol["f"] * rms, msg
    assert rel(out_w, ref["virial"]) <= tol["w"], msg


@pytest.mark.parametrize("L", [2, 4, 6, 8, 10, 12, 14, 16, 18, 20])
def test_level_table_bit_exact(gpu_lib, L):
    p = params(L, 1, 0)
    model = mtp.Model.from_params(p)
    assert model.level_table().tolist() == levels.level_table(L)
    assert model.m == len(levels.basis(L))


def _oracle_lists(cfg, rc):
    counts, j, s, d = oracle.neighbors(cfg.pos, cfg.cell, rc)
    return counts, j, s, d


def test_neighbors_bit_exact_single_and_batched(gpu_lib):
    rng = np.random.default_rng(17)
    cfgs = [synth.bcc_128()]
    cfgs += [synth.random_small_config(rng, 8, 96) for _ in range(20)]
    # a one-atom cell and a thin triclinic cell (many images)
    cfgs.append(synth.Config(np.array([[0.3, 0.2, 0.1]]), np.zeros(1, np.int32), np.diag([2.6, 2.9, 3.1])))
    thin = synth.Config(rng.normal(0, 0.4, (3, 3)) + 1.0, np.zeros(3, np.int32),
                        np.array([[3.0, 0, 0], [1.4, 2.7, 0], [0.6, 0.9, 2.2]]))
    cfgs.append(thin)
    b = synth.pack(cfgs)
    for c in cfgs:
        c.types[:] = 0
    b.types[:] = 0
    model = mtp.Model.from_params(params(8, 1, 0))
    pos, types, cells, off = batch_tensors(b)
    counts, j, s, r = model.neighbors(pos, cells, off)
    counts, j, s, r = counts.cpu().numpy(), j.cpu().numpy(), s.cpu().numpy(), r.cpu().numpy()
    q = 0
    for k, c in enumerate(cfgs):
        oc, oj, os_, od = _oracle_lists(c, 5.0)
        a0, a1 = b.cfg_off[k], b.cfg_off[k + 1]
        np.testing.assert_array_equal(counts[a0:a1], oc)
        P = int(oc.sum())
        np.testing.assert_array_equal(j[q:q + P] - a0, oj)
        np.testing.assert_array_equal(s[q:q + P], os_)
        assert np.array_equal(r[q:q + P], od), "r_ij must be bit-identical"
        q += P


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_config1_bcc128_lev10(gpu_lib, precision):
    cfg = synth.bcc_128()
    p = params(10, 1, 1)
    ref = oracle.Potential(p).eval(cfg, want_b=True)
    model = mtp.Model.from_params(p, precision)
    out = model.eval(dev(cfg.pos, torch.float64), dev(cfg.types, torch.int32), dev(cfg.cell, torch.float64),
                     site=True, b_rows=True)
    tol = TOL[precision]
    check_config(out["energy"].item(), out["forces"].cpu().numpy(), out["virial"].cpu().numpy(), ref, cfg.n, tol)
    np.testing.assert_allclose(out["site"].cpu().numpy(), ref["site"], rtol=tol["e"] * 10,
                               atol=tol["e"] * np.abs(ref["site"]).max())
    np.testing.assert_allclose(out["b_rows"].cpu().numpy(), ref["b_atoms"].sum(0), rtol=tol["e"] * 10,
                               atol=tol["e"] * np.abs(ref["b_atoms"].sum(0)).max())
    # finite-difference check of the device forces (central differences of the device energy)
    if precision == "fp64":
        h = 1e-5
        F = out["forces"].cpu().numpy()
        rms = np.sqrt(np.mean(F ** 2))
        for i, k in [(0, 0), (17, 1), (101, 2)]:
            pp = cfg.pos.copy()
            pp[i, k] += h
            pm = cfg.pos.copy()
            pm[i, k] -= h
            ep = model.eval(dev(pp, torch.float64), dev(cfg.types, torch.int32), dev(cfg.cell, torch.float64))
            em = model.eval(dev(pm, torch.float64), dev(cfg.types, torch.int32), dev(cfg.cell, torch.float64))
            fd = -(ep["energy"].item() - em["energy"].item()) / (2 * h)
            assert abs(fd - F[i, k]) <= 1e-7 * rms


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [12, 16])
def test_batched_small_cells(gpu_lib, precision, L):
    b = synth.small_cells(n_cfg=24, n_lo=8, n_hi=150, seed=30 + L)
    p = params(L, 3, 7)
    pot = oracle.Potential(p)
    model = mtp.Model.from_params(p, precision)
    pos, types, cells, off = batch_tensors(b)
    out = model.eval_batch(pos, types, cells, off, site=True, b_rows=True)
    e = out["energy"].cpu().numpy()
    f = out["forces"].cpu().numpy()
    w = out["virial"].cpu().numpy()
    br = out["b_rows"].cpu().numpy()
    tol = TOL[precision]
    for k in range(b.n_cfg):
        c = b.config(k)
        ref = pot.eval(c, want_b=True)
        a0, a1 = b.cfg_off[k], b.cfg_off[k + 1]
        check_config(e[k], f[a0:a1], w[k], ref, c.n, tol, msg=f"cfg {k}")
        rb = ref["b_atoms"].sum(0)
        assert rel(br[k], rb) <= tol["e"] * 10, f"b row {k}"
    # sum of site energies equals the configuration energies
    site = out["site"].cpu().numpy()
    for k in range(b.n_cfg):
        assert site[b.cfg_off[k]:b.cfg_off[k + 1]].sum() == pytest.approx(e[k], rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_threads_per_atom_variants(gpu_lib, precision):
    """Every lanes-per-atom layout of the pair kernels gives the oracle's results; changing the
    layout between two identical calls is honoured (the captured graph is dropped)."""
    L = 12
    b = synth.small_cells(n_cfg=10, n_lo=8, n_hi=120, seed=77)
    p = params(L, 3, 9)
    pot = oracle.Potential(p)
    refs = [pot.eval(b.config(k)) for k in range(b.n_cfg)]
    model = mtp.Model.from_params(p, precision)
    pos, types, cells, off = batch_tensors(b)
    tol = TOL[precision]
    out = None
    for tm, tp in [(1, 1), (2, 4), (4, 2), (8, 8), (1, 8), (8, 1), (0, 0)]:
        model.set_threads_per_atom(tm, tp)
        for _ in range(2):  # the second identical call replays a graph
            out = model.eval_batch(pos, types, cells, off, out=out)
            e, f, w = (out[k].cpu().numpy() for k in ("energy", "forces", "virial"))
            for k in range(b.n_cfg):
                a0, a1 = b.cfg_off[k], b.cfg_off[k + 1]
                check_config(e[k], f[a0:a1], w[k], refs[k], b.config(k).n, tol, msg=f"tpa {tm},{tp} cfg {k}")
    with pytest.raises(mtp.MTPError):
        model.set_threads_per_atom(3, 1)


@pytest.fixture(scope="module")
def config2():
    cfg = synth.fcc_binary()
    assert cfg.n == 16384
    p = params(16, 2, 2)
    return cfg, p, oracle.Potential(p).eval(cfg)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_config2_fcc16_lev16_full(gpu_lib, config2, precision):
    """16,384-atom fcc binary alloy at lev_max 16 against the full oracle evaluation."""
    cfg, p, ref = config2
    model = mtp.Model.from_params(p, precision)
    out = model.eval(dev(cfg.pos, torch.float64), dev(cfg.types, torch.int32), dev(cfg.cell, torch.float64),
                     site=True)
    site = out["site"].cpu().numpy()
    F = out["forces"].cpu().numpy()
    tol = TOL[precision]
    check_config(out["energy"].item(), F, out["virial"].cpu().numpy(), ref, cfg.n, tol)
    assert out["energy"].item() == pytest.approx(site.sum(), rel=1e-9)
    # site energies at the energy bar, relative to each site's energy (never below the per-atom
    # energy scale RMS(V))
    scale = np.maximum(np.abs(ref["site"]), np.sqrt(np.mean(ref["site"] ** 2)))
    worst = np.max(np.abs(site - ref["site"]) / scale)
    assert worst <= tol["e"], worst
    rms_f = np.sqrt(np.mean(F ** 2))
    assert np.abs(F.sum(0)).max() <= (1e-9 if precision == "fp64" else 1e-3) * rms_f * np.sqrt(cfg.n)


def test_edge_cases(gpu_lib):
    p = params(8, 2, 3)
    model = mtp.Model.from_params(p)
    pot = oracle.Potential(p)
    # a batch with an empty configuration and a single-atom cell (self images only)
    one = synth.Config(np.array([[0.1, 0.2, 0.3]]), np.array([1], np.int32), np.diag([3.1, 2.8, 3.3]))
    empty = synth.Config(np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 4.0)
    rng = np.random.default_rng(4)
    odd = synth.random_small_config(rng, 33, 33, species_pool=(0, 1), max_species=2)
    b = synth.pack([one, empty, odd])
    pos, types, cells, off = batch_tensors(b)
    out = model.eval_batch(pos, types, cells, off)
    e = out["energy"].cpu().numpy()
    assert e[1] == 0.0
    for k, c in ((0, one), (2, odd)):
        ref = pot.eval(c)
        assert e[k] == pytest.approx(ref["energy"], rel=1e-10)
    # invalid species -> EINVAL
    bad = types.clone()
    bad[0] = 5
    with pytest.raises(mtp.MTPError) as ei:
        model.eval_batch(pos, bad, cells, off)
    assert ei.value.code == 1
    # capacity overflow -> EOVERFLOW, then a larger capacity succeeds
    model.set_neighbor_capacity(8)
    with pytest.raises(mtp.MTPError) as ei:
        model.eval_batch(pos, types, cells, off)
    assert ei.value.code == 4
    model.set_neighbor_capacity(128)
    out2 = model.eval_batch(pos, types, cells, off)
    np.testing.assert_allclose(out2["energy"].cpu().numpy(), e, rtol=1e-12)


def test_host_memory_path_matches_device_path(gpu_lib):
    b = synth.small_cells(n_cfg=6, n_lo=16, n_hi=64, seed=9)
    p = params(10, 3, 4)
    model = mtp.Model.from_params(p, "fp32")
    pos, types, cells, off = batch_tensors(b)
    ref = model.eval_batch(pos, types, cells, off)
    K, N = b.n_cfg, b.n_atoms
    e = np.zeros(K)
    f = np.zeros((N, 3))
    w = np.zeros((K, 9))
    mtp.mtp_eval_batch(model.h, K, N, b.cfg_off, b.pos, b.types, b.cells.reshape(K, 9), e, f, w,
                       flags=mtp.HOST_MEMORY)
    # the per-configuration sums use double-precision atomics, so the order of additions may differ
    np.testing.assert_allclose(e, ref["energy"].cpu().numpy(), rtol=1e-13)
    np.testing.assert_allclose(f, ref["forces"].cpu().numpy(), rtol=1e-6, atol=1e-6 * np.abs(f).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replay_tracks_new_inputs(gpu_lib, precision):
    """Repeated identical calls replay a captured CUDA graph; the graph must read the current values."""
    cfg = synth.bcc_128()
    p = params(10, 1, 1)
    model = mtp.Model.from_params(p, precision)
    pos = dev(cfg.pos, torch.float64)
    types, cells = dev(cfg.types, torch.int32), dev(cfg.cell.reshape(1, 3, 3), torch.float64)
    off = dev(np.array([0, cfg.n]), torch.int32)
    out = None
    rng = np.random.default_rng(5)
    for k in range(5):
        moved = cfg.pos + rng.normal(0, 0.02, size=cfg.pos.shape)
        pos.copy_(dev(moved, torch.float64))  # same buffer, new values
        out = model.eval_batch(pos, types, cells, off, out=out)
        ref = mtp.Model.from_params(p, precision).eval_batch(pos, types, cells, off)
        assert out["energy"].item() == pytest.approx(ref["energy"].item(), rel=1e-12)
        np.testing.assert_allclose(out["forces"].cpu().numpy(), ref["forces"].cpu().numpy(), rtol=1e-12,
                                   atol=1e-12 * np.abs(ref["forces"].cpu().numpy()).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [18, 20])
def test_batched_small_cells_high_level(gpu_lib, precision, L):
    """lev_max 18 and 20 (straight-line contraction with spills in the float path), scaled parameters."""
    b = synth.small_cells(n_cfg=6, n_lo=12, n_hi=40, seed=60 + L)
    p = synth.scaled_params(L, 3, 8, 2.0, 5.0, synth.labels_from_level_table(levels.level_table(L)), seed=61)
    pot = oracle.Potential(p)
    model = mtp.Model.from_params(p, precision)
    pos, types, cells, off = batch_tensors(b)
    out = model.eval_batch(pos, types, cells, off, b_rows=True)
    e, f, w = out["energy"].cpu().numpy(), out["forces"].cpu().numpy(), out["virial"].cpu().numpy()
    br = out["b_rows"].cpu().numpy()
    tol = TOL[precision]
    for k in range(b.n_cfg):
        ref = pot.eval(b.config(k), want_b=True)
        a0, a1 = b.cfg_off[k], b.cfg_off[k + 1]
        check_config(e[k], f[a0:a1], w[k], ref, b.config(k).n, tol, msg=f"cfg {k}")
        assert rel(br[k], ref["b_atoms"].sum(0)) <= tol["e"] * 10
