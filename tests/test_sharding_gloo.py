"""Particle-id sharding across ranks (the multi-GPU layout: replicated
geometry, contiguous id ranges, one integer all-reduce of the tallies),
exercised with world_size 2 on CPU ranks over gloo: each rank tracks its id
range (with the oracle, the one tracker that runs without a GPU) and the
product's merge (paper_2406_13849_gb300.sharding) combines them.  Integer
sums make the merged tally independent of the partition: it must equal the
single-rank run bit for bit.  The library's own sharded runs are compared
with the whole run on the GPU (tests/test_gpu_sharding.py)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import sharding as S

N_TOTAL = 1601


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out, plant_status):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = O.Geometry(I.to_json(I.small_core()), O.MODE_CSG)
    first, n = S.shard_range(N_TOTAL, rank, world)
    r = g.run(n, 3, 0.25, first_id=first, records=False)
    t = torch.from_numpy(r["tally"].view(np.int64).copy())
    c = torch.from_numpy(r["counters"].view(np.int64).copy())
    if plant_status and rank == 1:
        c[S.STATUS] = -7          # a kernel-level status on one rank only
    S.merge_tallies(t, c)
    if rank == 0:
        np.save(out, np.concatenate([t.numpy(), c.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_sum_to_single_run(tmp_path):
    out = str(tmp_path / "merged.npy")
    mp.spawn(_rank, args=(2, _free_port(), out, False), nprocs=2, join=True)
    merged = np.load(out).view(np.uint64)
    g = O.Geometry(I.to_json(I.small_core()), O.MODE_CSG)
    whole = g.run(N_TOTAL, 3, 0.25, records=False)
    ni = g.n_inst
    assert np.array_equal(merged[:ni], whole["tally"])
    assert np.array_equal(merged[ni:], whole["counters"])


def test_merge_keeps_a_status_any_rank_reported(tmp_path):
    out = str(tmp_path / "merged.npy")
    mp.spawn(_rank, args=(2, _free_port(), out, True), nprocs=2, join=True)
    merged = np.load(out)
    assert merged[-16 + S.STATUS] == -7


def test_shard_range_covers_ids_once():
    for n, w in ((0, 3), (7, 3), (1601, 2), (10_000_000, 8)):
        ranges = [S.shard_range(n, r, w) for r in range(w)]
        assert sum(c for _, c in ranges) == n
        assert all(ranges[r][0] + ranges[r][1] == ranges[r + 1][0] for r in range(w - 1))
        assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1


def test_shard_geometries_balances_particles():
    counts = [int(c) for _, c in I.config4()]
    for w in (1, 2, 4, 8):
        parts = S.shard_geometries(counts, w)
        assert sorted(k for p in parts for k in p) == list(range(len(counts)))
        loads = [sum(counts[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(counts)
