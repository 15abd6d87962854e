"""Splitting one database across GPUs (one process per GPU).

Database sequences are independent alignment problems (the paper's inter-task scheme), so a
database shards with no exchange during the search: rank r loads `shard_indices(...)[r]`,
searches it on its own GPU, and the per-rank scores are put back in original order by
`merge_scores`.  Sequences are dealt longest first to the rank holding the fewest residues,
which balances the cell counts (and so the search times) across ranks.
"""

from __future__ import annotations

import heapq

import numpy as np


def shard_indices(offsets, world_size: int) -> list:
    """Original sequence indices of each rank's shard (each sorted ascending)."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    lens = np.diff(np.asarray(offsets, dtype=np.int64))
    order = np.argsort(-lens, kind="stable")
    heap = [(0, r) for r in range(world_size)]
    parts = [[] for _ in range(world_size)]
    for k in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(k))
        heapq.heappush(heap, (load + int(lens[k]), r))
    return [np.sort(np.array(p, dtype=np.int64)) for p in parts]


def shard_database(residues, offsets, indices):
    """(residues, offsets) of the sequences `indices`, in that order."""
    offsets = np.asarray(offsets, dtype=np.int64)
    idx = np.asarray(indices, dtype=np.int64)
    lens = offsets[idx + 1] - offsets[idx]
    new_off = np.zeros(idx.shape[0] + 1, dtype=np.int64)
    np.cumsum(lens, out=new_off[1:])
    out = np.empty(int(new_off[-1]), dtype=np.uint8)
    res = np.asarray(residues)
    for t, k in enumerate(idx):
        out[new_off[t]:new_off[t + 1]] = res[offsets[k]:offsets[k + 1]]
    return out, new_off


def merge_scores(num_seqs: int, parts, part_scores) -> np.ndarray:
    """Scores in original order from per-rank (indices, scores[..., len(indices)]) pairs."""
    first = np.asarray(part_scores[0])
    out = np.zeros(first.shape[:-1] + (int(num_seqs),), dtype=first.dtype)
    for idx, sc in zip(parts, part_scores):
        out[..., np.asarray(idx, dtype=np.int64)] = sc
    return out
