"""Writes the stored expected scores of the full-size parity tests, from the oracle alone.

    python tests/golden/make_fullsize_golden.py batched [--threads N]
    python tests/golden/make_fullsize_golden.py long_subject [--pairs 2000]
    python tests/golden/make_fullsize_golden.py paper_shaped [--pairs 1200]

Every value comes from ``oracle`` (the int64 CPU recurrence of Eqs. sw2-sw4) on the seeded
inputs of ``workloads``; nothing here runs or reads the CUDA path.  Run it on the CPU, once.

``batched`` (20 queries, 144..5478 residues, vs the 1M-sequence database: 7.66e12 cells, a
few hours on 8 cores) scores EVERY (query, sequence) pair and stores, per query row, the
SHA-256 of the row as little-endian int32, its maximum and first argmax, and the SHA-256 of
each block of ``BLOCK`` consecutive scores (first 16 hex digits), so a test can name the block
of a mismatch and recompute only that block.  Rows finished so far are kept in a partial file
and the run resumes from it.

``long_subject`` (5 queries vs 50,000 subjects of 5,000..35,000 residues) and
``paper_shaped`` (the 20 queries vs 6M sequences) -- 1.3e13 and 4.6e13 cells, too many for a
full pass -- store the exact scores of a seeded sample of pairs: the 50 (20) longest subjects
against every query, then random pairs.

Each file also records fingerprints of the inputs (SHA-256 of the residues, offsets, queries
and matrix), so a test can tell a changed generator from a wrong score.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as w  # noqa: E402

BLOCK = 16384
GOE, GE = 10, 2


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def fingerprints(wl) -> dict:
    return {"residues": sha(wl.db.residues), "offsets": sha(wl.db.offsets.astype("<i8")),
            "queries": [sha(q) for q in wl.queries], "matrix": sha(wl.matrix.astype(np.int8)),
            "num_seqs": wl.db.num_seqs, "num_residues": wl.db.num_residues,
            "query_lengths": [len(q) for q in wl.queries], "gap_open": GOE, "gap_extend": GE}


def row_record(scores: np.ndarray) -> dict:
    row = scores.astype("<i4")
    return {"sha256": sha(row), "max": int(row.max()) if row.size else 0,
            "argmax": int(np.argmax(row)) if row.size else -1,
            "blocks": [sha(row[b:b + BLOCK])[:16] for b in range(0, row.size, BLOCK)]}


def make_batched(threads: int) -> str:
    out = os.path.join(HERE, "fullsize_batched.json")
    part = out + ".partial"
    wl = w.batched()
    fp = fingerprints(wl)
    done = {}
    if os.path.exists(part):
        with open(part) as f:
            prev = json.load(f)
        if prev.get("inputs") == fp:
            done = {int(k): v for k, v in prev["rows"].items()}
    order = sorted(range(len(wl.queries)), key=lambda k: len(wl.queries[k]))
    for k in order:
        if k in done:
            continue
        t0 = time.time()
        s, used = oracle.sw_search(wl.queries[k], wl.db.residues, wl.db.offsets, wl.matrix,
                                   GOE, GE, threads=threads)
        assert s.max() < 2 ** 31
        done[k] = row_record(s)
        dt = time.time() - t0
        print(f"query {k} (m={len(wl.queries[k])}): {dt:.0f} s on {used} threads, "
              f"{len(wl.queries[k]) * wl.db.num_residues / dt / 1e9:.2f} GCUPS", flush=True)
        with open(part + ".tmp", "w") as f:
            json.dump({"inputs": fp, "rows": {str(i): r for i, r in done.items()}}, f)
        os.replace(part + ".tmp", part)
    doc = {"what": "oracle scores of every (query, sequence) pair of the batched workload "
                   "(20 queries vs 1M sequences, gaps 10/2): per query row the SHA-256 of the "
                   "int32 row, its max, first argmax and SHA-256 prefixes of blocks of "
                   f"{BLOCK} scores",
           "written_by": "tests/golden/make_fullsize_golden.py batched (oracle only)",
           "block": BLOCK, "inputs": fp,
           "rows": [done[k] for k in range(len(wl.queries))]}
    with open(out, "w") as f:
        json.dump(doc, f, indent=0)
    os.remove(part)
    return out


def make_sampled(name: str, n_pairs: int, n_longest: int, threads: int, query_lengths=None) -> str:
    out = os.path.join(HERE, f"fullsize_{name}.json")
    wl = getattr(w, name)() if query_lengths is None else \
        getattr(w, name)(query_lengths=query_lengths)
    nq, n = len(wl.queries), wl.db.num_seqs
    lens = wl.db.lengths()
    rng = np.random.default_rng(np.random.SeedSequence([1702, 7195, len(name)]))
    pairs = set()
    for s in np.argsort(-lens, kind="stable")[:n_longest]:
        for q in range(nq):
            pairs.add((q, int(s)))
    while len(pairs) < n_pairs:
        pairs.add((int(rng.integers(nq)), int(rng.integers(n))))
    pairs = sorted(pairs)
    qsel = np.array([p[0] for p in pairs], np.int64)
    dsel = np.array([p[1] for p in pairs], np.int64)
    t0 = time.time()
    exp = oracle.sw_pairs(wl.queries, wl.db.residues, wl.db.offsets, qsel, dsel, wl.matrix,
                          GOE, GE, threads=threads)
    print(f"{name}: {len(pairs)} pairs in {time.time() - t0:.0f} s", flush=True)
    doc = {"what": f"oracle scores of a seeded sample of (query, sequence) pairs of the {name} "
                   f"workload (gaps 10/2): the {n_longest} longest subjects against every query, "
                   "then random pairs",
           "written_by": f"tests/golden/make_fullsize_golden.py {name} (oracle only)",
           "inputs": fingerprints(wl),
           "pairs": [[int(q), int(d), int(e)] for q, d, e in zip(qsel, dsel, exp)]}
    with open(out, "w") as f:
        json.dump(doc, f, separators=(",", ":"))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["batched", "long_subject", "paper_shaped"])
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--pairs", type=int, default=0)
    a = ap.parse_args()
    oracle.build()
    if a.workload == "batched":
        print(make_batched(a.threads))
    elif a.workload == "long_subject":
        print(make_sampled("long_subject", a.pairs or 2000, 50, a.threads))
    else:
        print(make_sampled("paper_shaped", a.pairs or 1200, 20, a.threads))


if __name__ == "__main__":
    main()
