"""The multi-GPU path on CPU: world size 2 over gloo.  Each rank takes its shard of one
database (shard_indices), scores it (the CPU oracle stands in for a rank's GPU), and rank 0
gathers the shards back into original order; the result equals the unsharded search.  The
benchmark's timing reduction (barrier, max over ranks) runs over the same process group.
No collective touches the data path of a search."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _load_shard_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_shard", os.path.join(ROOT, "paper_1702_07195_gb300", "shard.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, result_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shard = _load_shard_module()
    wl = w.plain(seed=3, scale=0.03)
    parts = shard.shard_indices(wl.db.offsets, world)
    res, offs = shard.shard_database(wl.db.residues, wl.db.offsets, parts[rank])
    mine, _ = oracle.sw_search(wl.queries[0], res, offs, wl.matrix, 10, 2, threads=1)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)          # bench.py's max-over-ranks timing
    dist.barrier()
    if rank == 0:
        merged = shard.merge_scores(wl.db.num_seqs, parts, gathered)
        full, _ = oracle.sw_search(wl.queries[0], wl.db.residues, wl.db.offsets, wl.matrix, 10, 2)
        np.save(result_path, np.stack([merged, full]))
        assert float(t.item()) == float(world)
    dist.destroy_process_group()


def test_sharded_search_world_size_2(tmp_path):
    path = str(tmp_path / "res.npy")
    mp.spawn(_rank, args=(2, _free_port(), path), nprocs=2, join=True)
    merged, full = np.load(path)
    assert np.array_equal(merged, full)


def test_shards_balance_and_cover():
    shard = _load_shard_module()
    wl = w.plain(seed=4, scale=0.2)
    for world in (1, 2, 3, 8):
        parts = shard.shard_indices(wl.db.offsets, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(wl.db.num_seqs))
        lens = np.diff(wl.db.offsets)
        loads = [int(lens[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= int(lens.max())
