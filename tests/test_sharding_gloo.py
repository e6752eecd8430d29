"""Particle-id sharding across ranks (the multi-GPU layout: replicated
geometry, contiguous id ranges, one integer all-reduce of the tallies),
exercised with world_size 2 on CPU ranks over gloo with the oracle as the
per-rank tracker.  Integer sums make the merged tally independent of the
partition: it must equal the single-rank run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2406_13849_gb300 import inputs as I

N_TOTAL = 1600


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = O.Geometry(I.to_json(I.small_core()), O.MODE_CSG)
    n = N_TOTAL // world
    r = g.run(n, 3, 0.25, first_id=rank * n, records=False)
    t = torch.from_numpy(r["tally"].view(np.int64).copy())
    c = torch.from_numpy(r["counters"].view(np.int64).copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out, np.concatenate([t.numpy(), c.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_sum_to_single_run(tmp_path):
    out = str(tmp_path / "merged.npy")
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    merged = np.load(out).view(np.uint64)
    g = O.Geometry(I.to_json(I.small_core()), O.MODE_CSG)
    whole = g.run(N_TOTAL, 3, 0.25, records=False)
    ni = g.n_inst
    assert np.array_equal(merged[:ni], whole["tally"])
    assert np.array_equal(merged[ni:], whole["counters"])
