"""Parity at full workload sizes, in the launch configuration bench.py times
(sw_search_batch_device on device buffers, autotuned kernel variant): every score is checked
by properties that hold at any size, and a seeded sample of (query, sequence) pairs -- the
longest sequences and the highest scores included -- is recomputed one by one by the oracle
and must match bit for bit."""

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_lib()
    import paper_1702_07195_gb300 as m
    return m


def _run_like_bench(sw, wl, tune=True):
    import torch
    nq = len(wl.queries)
    cat = np.concatenate(wl.queries)
    qoff = np.zeros(nq + 1, np.int64)
    np.cumsum([len(q) for q in wl.queries], out=qoff[1:])
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as db:
        if tune and nq >= 2:
            srt = sorted(wl.queries, key=len)
            sw.sw_db_tune(db, srt[len(srt) // 2 - 1: len(srt) // 2 + 1], wl.matrix, 10, 2)
        d_q = torch.from_numpy(cat).cuda()
        d_s = torch.empty(nq * db.num_seqs, dtype=torch.int32, device="cuda")
        for _ in range(2):   # the second run is a CUDA-graph replay, as in the timed steps
            sw.sw_search_batch_device(db, d_q, qoff, wl.matrix, 10, 2, d_s)
        torch.cuda.synchronize()
        st = sw.sw_get_stats(db)
        return d_s.cpu().numpy().reshape(nq, -1), st


def _check_sample(wl, got, n_random, seed, extra_pairs=()):
    nq, n = got.shape
    rng = np.random.default_rng(seed)
    lens = wl.db.lengths()
    pairs = set((int(rng.integers(nq)), int(rng.integers(n))) for _ in range(n_random))
    longest = np.argsort(-lens)[:3]
    for q in range(nq):
        pairs.add((q, int(np.argmax(got[q]))))         # the top hit of every query
    for s in longest:
        pairs.add((int(rng.integers(nq)), int(s)))
    pairs |= set(extra_pairs)
    pairs = sorted(pairs)
    qsel = np.array([p[0] for p in pairs], np.int64)
    dsel = np.array([p[1] for p in pairs], np.int64)
    exp = oracle.sw_pairs(wl.queries, wl.db.residues, wl.db.offsets, qsel, dsel, wl.matrix, 10, 2)
    bad = [(p, int(got[p]), int(e)) for p, e in zip(pairs, exp) if got[p] != e]
    assert not bad, f"{len(bad)} of {len(pairs)} sampled scores differ: {bad[:5]}"
    return len(pairs)


def _check_properties(wl, got):
    lens = wl.db.lengths()
    assert got.min() >= 0, "a negative score (unresolved saturation marker?)"
    maxs = int(wl.matrix.max())
    for q in range(got.shape[0]):
        bound = np.minimum(lens, len(wl.queries[q])) * maxs
        assert (got[q] <= bound).all()
        assert (got[q][lens == 0] == 0).all()


def test_batched_full_size(sw):
    """20 queries (144..5478) vs 1M sequences: the default benchmark workload."""
    wl = w.batched()
    got, st = _run_like_bench(sw, wl)
    assert st["multi_query"] == 1 and st["graph_replay"] == 1
    _check_properties(wl, got)
    assert _check_sample(wl, got, 300, seed=1) >= 300


def test_paper_shaped_full_size(sw):
    """20 queries vs 6M sequences (1.5G residues, lengths up to 35,000): inter-task kernel for
    the bulk, intra-task kernel for the subjects above the cutoff."""
    wl = w.paper_shaped(query_lengths=[144, 807, 5478])
    got, st = _run_like_bench(sw, wl)
    assert st["intra_ms"] > 0
    _check_properties(wl, got)
    _check_sample(wl, got, 200, seed=2)


def test_long_subject_full_size(sw):
    """5 queries (1,000..5,000) vs 50,000 subjects of 5,000..35,000 residues: all intra-task."""
    wl = w.long_subject()
    got, st = _run_like_bench(sw, wl, tune=False)
    assert st["inter_cells"] == 0 and st["intra_ms"] > 0
    _check_properties(wl, got)
    _check_sample(wl, got, 25, seed=3)
