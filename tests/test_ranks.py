"""Multi-rank host logic on CPU (gloo, world size 2): replicas are distinct, shards cover a batch
exactly once with balanced atom counts, and the job's time and throughput come from the slowest
rank.  No GPU and no data-path collective is involved: configurations are independent."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2007_08555_gb300 import ranks, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = ranks.env()
        assert (r, w, local) == (rank, world, rank)
        # replicas: the bench workload shape, a seed per rank
        cfg = synth.fcc_binary(reps=3, seed=ranks.replica_seed(2, r))
        digest = torch.tensor([float(np.sum(cfg.pos * np.arange(1, cfg.n + 1)[:, None]))], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(w)]
        dist.all_gather(gathered, digest)
        # shards of one batch, built identically on every rank
        b = synth.small_cells(n_cfg=37, n_lo=8, n_hi=64, seed=11)
        mine = ranks.local_batch(b, r, w)
        n_mine = ranks.sum_over_ranks(mine.n_atoms)
        k_mine = ranks.sum_over_ranks(mine.n_cfg)
        # timings: the slowest rank sets the job time
        t_max = ranks.max_over_ranks(1.5 + r)
        thr = ranks.job_throughput(ranks.sum_over_ranks(cfg.n), t_max)
        results[rank] = dict(digests=[float(g.item()) for g in gathered], n_mine=n_mine, k_mine=k_mine,
                             n_total=b.n_atoms, k_total=b.n_cfg, t_max=t_max, thr=thr, n_rep=cfg.n,
                             first_pos=mine.pos[0].tolist(), off0=int(mine.cfg_off[0]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    manager = mp.get_context("spawn").Manager()
    results = manager.dict()
    mp.start_processes(_worker, args=(world, _free_port(), results), nprocs=world, join=True, start_method="spawn")
    assert len(results) == world
    r0, r1 = results[0], results[1]
    assert r0["digests"] == r1["digests"]
    assert r0["digests"][0] != r0["digests"][1], "replicas must differ between ranks"
    for r in (r0, r1):
        assert r["n_mine"] == r["n_total"] and r["k_mine"] == r["k_total"]
        assert r["t_max"] == 2.5
        assert r["thr"] == pytest.approx(2 * r["n_rep"] / 2.5e-3)
        assert r["off0"] == 0


def test_shard_ranges_cover_and_balance():
    b = synth.small_cells(n_cfg=200, n_lo=8, n_hi=256, seed=5)
    for world in (1, 2, 3, 8):
        rg = ranks.shard_ranges(b.cfg_off, world)
        assert rg[0][0] == 0 and rg[-1][1] == b.n_cfg
        assert all(rg[k][1] == rg[k + 1][0] for k in range(world - 1))
        atoms = [int(b.cfg_off[k1] - b.cfg_off[k0]) for k0, k1 in rg]
        assert sum(atoms) == b.n_atoms
        # a cut misses its target by less than one configuration (at most 256 atoms)
        assert max(atoms) - min(atoms) <= 2 * 256
    # more ranks than configurations: empty ranges, still a cover
    small = synth.small_cells(n_cfg=2, n_lo=8, n_hi=16, seed=1)
    rg = ranks.shard_ranges(small.cfg_off, 4)
    assert sum(k1 - k0 for k0, k1 in rg) == 2


def test_local_batch_reassembles():
    b = synth.small_cells(n_cfg=50, n_lo=8, n_hi=64, seed=7)
    parts = [ranks.local_batch(b, r, 3) for r in range(3)]
    np.testing.assert_array_equal(np.concatenate([p.pos for p in parts]), b.pos)
    np.testing.assert_array_equal(np.concatenate([p.types for p in parts]), b.types)
    np.testing.assert_array_equal(np.concatenate([p.cells for p in parts]), b.cells)
    for p in parts:
        assert p.cfg_off[0] == 0 and p.cfg_off[-1] == p.n_atoms


def test_single_process_reductions_are_identity():
    assert ranks.max_over_ranks(3.0) == 3.0
    assert ranks.sum_over_ranks(4.0) == 4.0
    with pytest.raises(ValueError):
        ranks.job_throughput(10, 0.0)
