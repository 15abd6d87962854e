"""Serving (continuous batching): each result is the same alone and in the mix (tolerance 0,
integer scores), matches the oracle, and requests that arrive while others are in flight
join the running ticks."""

import threading
import time

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


def _db_with_long_and_saturation():
    wl = w.batched(seed=21, scale=0.004)
    db2, q_sat, _ = w.plant_saturating(wl.db, w.encode("MKTAYIAKQR"), count=3, run=3050)
    rng = np.random.default_rng(3)
    seqs = [db2.seq(i) for i in range(db2.num_seqs)] + [w.draw_residues(rng, 4100), w.draw_residues(rng, 5000)]
    return w.from_sequences(seqs), q_sat, wl.matrix


def test_alone_equals_mix_equals_oracle(sw):
    db, q_sat, sm = _db_with_long_and_saturation()
    qs = w.serving_queries(14, seed=4) + [q_sat, np.zeros(0, np.uint8)]
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, long_cutoff=4000) as h:
        with sw.Server(h, sm, 10, 2, max_inflight=6, slices=3) as srv:
            alone = [srv.wait(srv.submit(q)) for q in qs]           # one at a time
            tickets = [srv.submit(q) for q in qs]                    # all at once
            mix = [srv.wait(t) for t in tickets]
            st = srv.stats()
    for k, (a, b) in enumerate(zip(alone, mix)):
        assert np.array_equal(a, b), f"request {k}: alone != mix"
    for k in range(len(qs)):                                         # every request
        exp, _ = oracle.sw_search(qs[k], db.residues, db.offsets, sm, 10, 2)
        assert np.array_equal(mix[k].astype(np.int64), exp), f"request {k} vs oracle"
    assert int(mix[len(qs) - 2].max()) > 32767
    assert st["completed"] == 2 * len(qs) and st["max_in_flight"] >= 2
    assert st["joined_while_running"] >= 1


def test_arrivals_join_running_ticks(sw):
    """Requests submitted from another thread while the server is busy are admitted into the
    ongoing batch (continuous batching), and results still equal the one-query search."""
    wl = w.batched(seed=22, scale=0.01)
    qs = w.serving_queries(24, seed=9)
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        ref = sw.sw_search_batch(h, qs, wl.matrix, 10, 2)
        with sw.Server(h, wl.matrix, 10, 2, max_inflight=8, slices=8) as srv:
            tickets = [None] * len(qs)

            def producer():
                for i, q in enumerate(qs):
                    tickets[i] = srv.submit(q)
                    time.sleep(0.002)

            th = threading.Thread(target=producer)
            th.start()
            th.join()
            out = [srv.wait(t) for t in tickets]
            st = srv.stats(reset=True)
    for k in range(len(qs)):
        assert np.array_equal(out[k], ref[k]), f"request {k}"
        exp, _ = oracle.sw_search(qs[k], wl.db.residues, wl.db.offsets, wl.matrix, 10, 2)
        assert np.array_equal(out[k].astype(np.int64), exp), f"request {k} vs oracle"
    assert st["joined_while_running"] >= 1 and st["ticks"] >= 2
    assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0


def test_server_rejects_and_times_out(sw):
    wl = w.plain(seed=23, scale=0.05)
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        with pytest.raises(sw.SwError):
            sw.Server(h, wl.matrix, 20000, 2)                        # int16 path only
        with sw.Server(h, wl.matrix, 10, 2, max_query_len=256, max_pending=1) as srv:
            with pytest.raises(sw.SwError) as e:
                srv.submit(w.draw_residues(np.random.default_rng(1), 300))
            assert e.value.status == -1
            with pytest.raises(sw.SwError) as e:
                srv.submit(np.array([1, 2, 77], np.uint8))
            assert e.value.status == -2
            t = srv.submit(wl.queries[0])
            with pytest.raises(sw.SwError) as e:
                srv.wait(123456, timeout_ms=10)
            assert e.value.status == -1                              # unknown ticket
            got = srv.wait(t)
            exp, _ = oracle.sw_search(wl.queries[0], wl.db.residues, wl.db.offsets, wl.matrix, 10, 2)
            assert np.array_equal(got.astype(np.int64), exp)
    big = w.batched(seed=24, scale=0.05)
    with sw.sw_db_load(big.db.residues, big.db.offsets, w.ALPHABET_SIZE) as h:
        with sw.Server(h, big.matrix, 10, 2, max_inflight=2) as srv:
            rng = np.random.default_rng(2)
            tickets = [srv.submit(w.draw_residues(rng, 5000)) for _ in range(8)]
            with pytest.raises(sw.SwError) as e:       # 8 x 6e10 cells cannot finish in 1 ms
                srv.wait(tickets[-1], timeout_ms=1)
            assert e.value.status == -5
            for t in tickets:
                assert srv.wait(t).shape == (h.num_seqs,)


def test_concurrent_clients(sw):
    """Four client threads submit and wait at the same time; every result equals the
    single-query search of the same query (the mix of one- and multi-request ticks)."""
    wl = w.batched(seed=25, scale=0.008)
    qs = w.serving_queries(20, seed=13)
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        ref = sw.sw_search_batch(h, qs, wl.matrix, 10, 2)
        out = [None] * len(qs)
        errors = []
        with sw.Server(h, wl.matrix, 10, 2, max_inflight=6, slices=4) as srv:

            def client(ids):
                try:
                    for i in ids:
                        out[i] = srv.wait(srv.submit(qs[i]))
                except Exception as exc:   # surfaced below
                    errors.append(exc)

            threads = [threading.Thread(target=client, args=(list(range(c, len(qs), 4)),))
                       for c in range(4)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            st = srv.stats()
    assert not errors, errors
    for k in range(len(qs)):
        assert np.array_equal(out[k], ref[k]), f"request {k}"
        exp, _ = oracle.sw_search(qs[k], wl.db.residues, wl.db.offsets, wl.matrix, 10, 2)
        assert np.array_equal(out[k].astype(np.int64), exp), f"request {k} vs oracle"
    assert st["completed"] == len(qs)


def test_only_long_subjects(sw):
    """A database whose every sequence is above the inter-task cutoff: ticks run only the
    intra-task work (no interleaved groups), and results still equal the oracle."""
    rng = np.random.default_rng(29)
    db = w.database_from_lengths(rng, rng.integers(100, 300, size=20))
    sm = w.blosum62()
    qs = w.serving_queries(5, seed=31)
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, long_cutoff=64) as h:
        with sw.Server(h, sm, 10, 2, max_inflight=4) as srv:
            out = [srv.wait(t) for t in [srv.submit(q) for q in qs]]
    for k, q in enumerate(qs):
        exp, _ = oracle.sw_search(q, db.residues, db.offsets, sm, 10, 2)
        assert np.array_equal(out[k].astype(np.int64), exp), f"request {k}"
