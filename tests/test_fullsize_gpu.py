"""Parity at full workload sizes, in the launch configuration bench.py times
(sw_search_batch_device on device buffers, autotuned kernel variant).  Every score is checked
by properties that hold at any size; the headline workload's 20 x 1M scores are all compared
with the oracle's (stored per-row hashes written by tests/golden/make_fullsize_golden.py from
the oracle alone); the paper-shaped and long-subject workloads, too large for a full oracle
pass, are compared with stored oracle scores of their longest subjects against every query
and of seeded random pairs.  Tolerance 0 (integer scores)."""

import hashlib
import json
import os

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


def _golden(name, wl):
    """Stored oracle results of a full-size workload (written by tests/golden/
    make_fullsize_golden.py from the oracle alone), after checking they were made from these
    very inputs."""
    path = os.path.join(os.path.dirname(__file__), "golden", f"fullsize_{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        doc = json.load(f)
    fp = doc["inputs"]
    assert fp["num_seqs"] == wl.db.num_seqs and fp["num_residues"] == wl.db.num_residues
    assert fp["queries"] == [_sha(q) for q in wl.queries], "query generator changed"
    assert fp["residues"] == _sha(wl.db.residues), "database generator changed"
    assert fp["offsets"] == _sha(wl.db.offsets.astype("<i8"))
    assert fp["matrix"] == _sha(wl.matrix.astype(np.int8))
    return doc


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _check_rows(wl, got, doc):
    """Every score: each int32 row's SHA-256 against the oracle's.  A row that differs is
    narrowed to its blocks by the stored block hashes, and the first differing block is
    recomputed by the oracle to name the first wrong score."""
    blk = doc["block"]
    for q, rec in enumerate(doc["rows"]):
        row = np.ascontiguousarray(got[q], dtype="<i4")
        assert int(row.max()) == rec["max"] and int(np.argmax(row)) == rec["argmax"], \
            f"query {q}: max/argmax {int(row.max())}/{int(np.argmax(row))} vs oracle {rec['max']}/{rec['argmax']}"
        if _sha(row) == rec["sha256"]:
            continue
        bad = [b for b, h in zip(range(0, row.size, blk), rec["blocks"]) if _sha(row[b:b + blk])[:16] != h]
        b0 = bad[0]
        idx = np.arange(b0, min(row.size, b0 + blk), dtype=np.int64)
        exp = oracle.sw_pairs(wl.queries, wl.db.residues, wl.db.offsets,
                              np.full(idx.size, q, np.int64), idx, wl.matrix, 10, 2)
        wrong = np.nonzero(row[idx].astype(np.int64) != exp)[0]
        first = int(idx[wrong[0]]) if wrong.size else -1
        raise AssertionError(f"query {q} (m={len(wl.queries[q])}): {len(bad)} blocks of {blk} "
                             f"differ; first wrong score at sequence {first}: "
                             f"gpu {row[first] if first >= 0 else None} oracle "
                             f"{exp[wrong[0]] if wrong.size else None}")


def _check_pairs(got, doc):
    bad = [(q, d, int(got[q, d]), e) for q, d, e in doc["pairs"] if int(got[q, d]) != e]
    assert not bad, f"{len(bad)} of {len(doc['pairs'])} stored oracle scores differ: {bad[:5]}"
    return len(doc["pairs"])


def test_batched_full_size(sw):
    """20 queries (144..5478) vs 1M sequences, the headline workload: all 20,000,000 scores
    against the stored oracle rows."""
    wl = w.batched()
    got, st = _run_like_bench(sw, wl)
    assert st["multi_query"] == 1 and st["graph_replay"] == 1
    _check_properties(wl, got)
    doc = _golden("batched", wl)
    if doc is None:
        assert _check_sample(wl, got, 300, seed=1) >= 300
        pytest.skip("tests/golden/fullsize_batched.json absent: checked a sample only")
    _check_rows(wl, got, doc)


def test_paper_shaped_full_size(sw):
    """The 20 queries vs 6M sequences (1.5G residues, lengths up to 35,000): inter-task kernel
    for the bulk, intra-task kernel for the subjects above the cutoff; stored oracle scores of
    the 20 longest subjects against every query and of random pairs, and a fresh sample."""
    wl = w.paper_shaped()
    got, st = _run_like_bench(sw, wl)
    assert st["intra_ms"] > 0
    _check_properties(wl, got)
    _check_sample(wl, got, 50, seed=2)
    doc = _golden("paper_shaped", wl)
    if doc is None:
        pytest.skip("tests/golden/fullsize_paper_shaped.json absent: checked a sample only")
    assert _check_pairs(got, doc) >= 1000


def test_long_subject_full_size(sw):
    """5 queries (1,000..5,000) vs 50,000 subjects of 5,000..35,000 residues, all intra-task:
    stored oracle scores of the 50 longest subjects against every query and of random pairs
    (2,000 pairs)."""
    wl = w.long_subject()
    got, st = _run_like_bench(sw, wl, tune=False)
    assert st["inter_cells"] == 0 and st["intra_ms"] > 0
    _check_properties(wl, got)
    doc = _golden("long_subject", wl)
    if doc is None:
        _check_sample(wl, got, 25, seed=3)
        pytest.skip("tests/golden/fullsize_long_subject.json absent: checked a sample only")
    assert _check_pairs(got, doc) >= 2000
