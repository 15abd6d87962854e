"""GPU parity: every score from the CUDA path (through the C ABI) equals the CPU oracle's,
bit for bit (integer arithmetic: tolerance 0).

Sizes span several 64-sequence groups, 32-row strips, 256-row profile chunks and ragged
tails; edge cases cover empty inputs, length-1 inputs, gap-cost regimes (including
Goe < Ge and costs too large for the int16 path), asymmetric matrices, planted hits that
saturate int16 lanes (exact int32 rescore, Section 4.2), the rescore sweep when the
saturation list overflows, and subjects routed to the intra-task kernel.
"""

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


def _oracle_all(queries, db, matrix, goe, ge):
    return np.stack([oracle.sw_search(q, db.residues, db.offsets, matrix, goe, ge)[0]
                     for q in queries]) if len(queries) else np.zeros((0, db.num_seqs), np.int64)


def _check(got, exp, what=""):
    got = np.asarray(got, dtype=np.int64)
    assert got.shape == exp.shape, (got.shape, exp.shape)
    bad = np.argwhere(got != exp)
    if bad.size:
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches; first at {i}: gpu {got[i]} oracle {exp[i]}")


def test_plain_reduced(sw):
    wl = w.plain(seed=1, scale=0.2)                      # 2,000 sequences, m = 144
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as db:
        got = sw.sw_search(db, wl.queries[0], wl.matrix, wl.gap_open, wl.gap_extend)
        st = sw.sw_get_stats(db)
    _check(got[None], _oracle_all(wl.queries, wl.db, wl.matrix, 10, 2), "plain")
    # a small database: every group routed to the intra-task stage, which the events time
    assert st["cells"] == 144 * wl.db.num_residues and st["inter_ms"] + st["intra_ms"] > 0


@pytest.mark.parametrize("m", [1, 2, 7, 31, 32, 33, 63, 64, 65, 255, 256, 257, 300, 513])
def test_query_lengths_around_tiles(sw, m):
    rng = np.random.default_rng(m)
    lens = np.concatenate([rng.integers(1, 400, size=133), [1, 2, 7, 8, 9, 15, 16, 17, 0]])
    db = w.database_from_lengths(rng, lens)
    q = w.draw_residues(rng, m)
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        got = sw.sw_search(h, q, sm, 10, 2)
    _check(got[None], _oracle_all([q], db, sm, 10, 2), f"m={m}")


@pytest.mark.parametrize("goe,ge", [(10, 2), (12, 2), (0, 0), (3, 7), (5, 0), (1, 1), (40, 1),
                                    (16383, 16383), (20000, 3), (500000, 1)])
def test_gap_regimes(sw, goe, ge):
    rng = np.random.default_rng(goe * 7 + ge)
    db = w.database_from_lengths(rng, rng.integers(0, 200, size=150))
    qs = [w.draw_residues(rng, 90), w.draw_residues(rng, 37)]
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        got = sw.sw_search_batch(h, qs, sm, goe, ge)
    _check(got, _oracle_all(qs, db, sm, goe, ge), f"gaps {goe},{ge}")


def test_asymmetric_matrix_and_small_alphabet(sw):
    rng = np.random.default_rng(42)
    A = 5
    sm = rng.integers(-6, 12, size=(A, A)).astype(np.int8)
    lens = rng.integers(0, 120, size=200)
    offs = np.zeros(201, np.int64)
    np.cumsum(lens, out=offs[1:])
    db = w.Database(rng.integers(0, A, size=int(offs[-1])).astype(np.uint8), offs)
    qs = [rng.integers(0, A, size=n).astype(np.uint8) for n in (70, 5, 33)]
    with sw.sw_db_load(db.residues, db.offsets, A) as h:
        got = sw.sw_search_batch(h, qs, sm, 4, 1)
    _check(got, _oracle_all(qs, db, sm, 4, 1), "asymmetric")


def test_empty_query_and_sequences(sw):
    rng = np.random.default_rng(3)
    db = w.database_from_lengths(rng, [0, 5, 0, 17, 1, 0])
    sm = w.blosum62()
    q = w.draw_residues(rng, 12)
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        got = sw.sw_search_batch(h, [np.zeros(0, np.uint8), q], sm, 10, 2)
    assert (got[0] == 0).all()
    _check(got[1:], _oracle_all([q], db, sm, 10, 2), "empty")


def test_single_sequence_database(sw):
    rng = np.random.default_rng(4)
    db = w.database_from_lengths(rng, [77])
    q = w.draw_residues(rng, 50)
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        got = sw.sw_search(h, q, sm, 10, 2)
    _check(got[None], _oracle_all([q], db, sm, 10, 2), "single")


def test_empty_database(sw):
    with sw.sw_db_load(np.zeros(0, np.uint8), np.array([0], np.int64), 24) as h:
        got = sw.sw_search(h, w.encode("MKV"), w.blosum62(), 10, 2)
    assert got.shape == (0,)


@pytest.mark.parametrize("flag_cap", [0, 2, 1])
def test_saturating_hits_rescored_exactly(sw, flag_cap, monkeypatch):
    """Planted hits above the int16 range go through the inter-task kernel (cutoff 8192, no
    routing of long groups), are flagged and rescored in int32; flag_cap 1 and 2 overflow the
    saturation list and exercise the sweep over all scores."""
    monkeypatch.setenv("SWGB_GROUP_SPLIT", "1000000000")
    wl = w.plain(seed=2, scale=0.05)
    db2, q2, idx = w.plant_saturating(wl.db, wl.queries[0], count=6, run=3200)
    with sw.sw_db_load(db2.residues, db2.offsets, w.ALPHABET_SIZE, long_cutoff=8192,
                       flag_cap=flag_cap) as h:
        got = sw.sw_search_batch(h, [q2, q2[:100], q2[-3300:]], wl.matrix, 10, 2)
        st = sw.sw_get_stats(h)
    exp = _oracle_all([q2, q2[:100], q2[-3300:]], db2, wl.matrix, 10, 2)
    _check(got, exp, "saturating")
    assert exp[0][idx].max() > 32767 and st["flagged"] >= 6


@pytest.mark.parametrize("block", ["1", "0"])
def test_long_subjects_intra_kernel(sw, block, monkeypatch):
    """Subjects above the cutoff on the int32 intra-task kernel: the block-shared-profile
    variant (default) and the per-warp variant (SWGB_INTRA_BLOCK=0); the packed int16x2
    wavefront kernel, which a batch of queries would otherwise take, is switched off."""
    monkeypatch.setenv("SWGB_INTRA_BLOCK", block)
    monkeypatch.setenv("SWGB_WAVE", "0")
    rng = np.random.default_rng(9)
    lens = np.concatenate([rng.integers(1, 300, size=120), rng.integers(1000, 2600, size=9), [4097]])
    db = w.database_from_lengths(rng, lens)
    qs = [w.draw_residues(rng, n) for n in (300, 1, 700)]
    sm = w.blosum62()
    exp = _oracle_all(qs, db, sm, 10, 2)
    for cutoff in (64, 512, 8192):
        with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, long_cutoff=cutoff) as h:
            got = sw.sw_search_batch(h, qs, sm, 10, 2)
        _check(got, exp, f"cutoff {cutoff}")


def test_long_subject_saturation(sw):
    """A long subject (intra-task int32 path) with a hit far above the int16 range."""
    run = np.full(4000, w.CODE_W, np.uint8)
    db = w.from_sequences([run, w.encode("WWWW"), run[:100]])
    q = np.concatenate([w.encode("MK"), run[:3500]])
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, long_cutoff=512) as h:
        got = sw.sw_search(h, q, w.blosum62(), 10, 2)
    assert got.tolist() == [3500 * 11, 44, 1100]


def test_batched_many_queries(sw):
    wl = w.batched(seed=5, scale=0.002, query_lengths=[144, 211, 375, 807, 1434])
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        got = sw.sw_search_batch(h, wl.queries, wl.matrix, 10, 2)
    _check(got, _oracle_all(wl.queries, wl.db, wl.matrix, 10, 2), "batched")


def test_device_api_torch_stream(sw):
    import torch
    wl = w.plain(seed=6, scale=0.03)
    qs = [wl.queries[0], wl.queries[0][:50]]
    cat = np.concatenate(qs)
    offs = np.array([0, len(qs[0]), len(cat)], np.int64)
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        dq = torch.from_numpy(cat).cuda()
        out = torch.full((2 * h.num_seqs,), -7, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            sw.sw_search_batch_device(h, dq, offs, wl.matrix, 10, 2, out, stream=s)
        s.synchronize()
        got = out.cpu().numpy().reshape(2, -1)
        # a repeated call with the same shapes and pointers
        out.fill_(-7)
        sw.sw_search_batch_device(h, dq, offs, wl.matrix, 10, 2, out)
        torch.cuda.synchronize()
        got2 = out.cpu().numpy().reshape(2, -1)
    exp = _oracle_all(qs, wl.db, wl.matrix, 10, 2)
    _check(got, exp, "device api")
    _check(got2, exp, "device api repeat")


def test_errors_are_reported(sw):
    rng = np.random.default_rng(1)
    db = w.database_from_lengths(rng, [10, 20])
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        with pytest.raises(sw.SwError) as e:
            sw.sw_search(h, np.array([1, 2, 99], np.uint8), w.blosum62(), 10, 2)
        assert e.value.status == -2
        with pytest.raises(sw.SwError) as e:
            sw.sw_search(h, np.array([1, 2], np.uint8), w.blosum62(), -1, 2)
        assert e.value.status == -1
        ok = sw.sw_search(h, w.draw_residues(rng, 30), w.blosum62(), 10, 2)
        assert ok.shape == (2,)
    with pytest.raises(sw.SwError) as e:
        sw.sw_db_load(np.array([0, 50], np.uint8), np.array([0, 2], np.int64), 24)
    assert e.value.status == -2


def test_results_independent_of_routing(sw):
    """Same scores whatever the inter/intra cutoff (property at any size)."""
    wl = w.plain(seed=8, scale=0.1)
    outs = []
    for cutoff in (128, 256, 3072):
        with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE, long_cutoff=cutoff) as h:
            outs.append(sw.sw_search(h, wl.queries[0], wl.matrix, 10, 2))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_every_kernel_variant_and_autotuner(sw, tmp_path):
    """Each inter-task variant (rows per strip x warps per block) gives the oracle's scores;
    the autotuner picks one, stores it in the cache and reuses it from there."""
    wl = w.batched(seed=12, scale=0.004, query_lengths=[100, 333, 700])
    exp = _oracle_all(wl.queries, wl.db, wl.matrix, 10, 2)
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        for v in range(4):
            sw.sw_db_set_variant(h, v)
            got = sw.sw_search_batch(h, wl.queries, wl.matrix, 10, 2)
            assert sw.sw_get_stats(h)["variant"] == v
            _check(got, exp, f"variant {v}")
        cache = str(tmp_path / "tune.txt")
        r1 = sw.sw_db_tune(h, [wl.queries[1]], wl.matrix, 10, 2, cache_path=cache)
        assert not r1["from_cache"] and r1["rows_per_strip"] in (32, 64)
        assert sum(g > 0 for g in r1["gcups"]) >= 2
        r2 = sw.sw_db_tune(h, [wl.queries[1]], wl.matrix, 10, 2, cache_path=cache)
        assert r2["from_cache"] and r2["variant"] == r1["variant"]
        got = sw.sw_search_batch(h, wl.queries, wl.matrix, 10, 2)
        assert sw.sw_get_stats(h)["variant"] == r1["variant"]
    _check(got, exp, "tuned")


def test_graph_replay_tracks_query_contents(sw):
    """A replayed graph rebuilds the query profile from the buffer's current contents."""
    import torch
    wl = w.plain(seed=13, scale=0.03)
    rng = np.random.default_rng(5)
    q1, q2 = w.draw_residues(rng, 120), w.draw_residues(rng, 120)
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        dq = torch.from_numpy(q1).cuda()
        out = torch.empty(h.num_seqs, dtype=torch.int32, device="cuda")
        offs = np.array([0, 120], np.int64)
        sw.sw_search_batch_device(h, dq, offs, wl.matrix, 10, 2, out)
        torch.cuda.synchronize()
        a = out.cpu().numpy().copy()
        dq.copy_(torch.from_numpy(q2))
        sw.sw_search_batch_device(h, dq, offs, wl.matrix, 10, 2, out)
        torch.cuda.synchronize()
        assert sw.sw_get_stats(h)["graph_replay"] == 1
        b = out.cpu().numpy().copy()
    _check(a[None], _oracle_all([q1], wl.db, wl.matrix, 10, 2), "first")
    _check(b[None], _oracle_all([q2], wl.db, wl.matrix, 10, 2), "replayed")


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_multi_query_kernel_matches_oracle(sw, variant, monkeypatch):
    """Two queries per register (multi-query kernel): ragged query lengths around the strip
    height, an empty query in the batch, an odd count, and planted int16 saturation, for every
    variant; the same batch with the multi-query path switched off agrees."""
    monkeypatch.setenv("SWGB_GROUP_SPLIT", "1000000000")   # keep every group on the int16 path
    rng = np.random.default_rng(100 + variant)
    base = w.batched(seed=14, scale=0.003).db
    db2, q_sat, _ = w.plant_saturating(base, w.draw_residues(rng, 20), count=3, run=3100)
    lens = [31, 32, 33, 0, 63, 65, 200, 1, 129]
    qs = [w.draw_residues(rng, n) for n in lens] + [q_sat]
    sm = w.blosum62()
    exp = _oracle_all(qs, db2, sm, 10, 2)
    with sw.sw_db_load(db2.residues, db2.offsets, w.ALPHABET_SIZE, long_cutoff=4096) as h:
        sw.sw_db_set_variant(h, variant)
        got = sw.sw_search_batch(h, qs, sm, 10, 2)
        st = sw.sw_get_stats(h)
        assert st["multi_query"] == 1 and st["flagged"] >= 3
        _check(got, exp, f"multi-query variant {variant}")
        monkeypatch.setenv("SWGB_MQ", "0")
        got2 = sw.sw_search_batch(h, qs, sm, 10, 2)
        assert sw.sw_get_stats(h)["multi_query"] == 0
    _check(got2, exp, "single-query kernel")


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1])
def test_multi_query_many_short_queries(sw, variant, seed, monkeypatch):
    """A batch of twenty-one queries, most shorter than one strip (lengths around 16-row
    multiples, two of length 1, one empty) plus a saturating query (int32 rescore): many
    query boundaries in both streams of the multi-query kernel, for every variant; every score
    equals the oracle."""
    monkeypatch.setenv("SWGB_GROUP_SPLIT", "1000000000")   # keep every group on the int16 path
    rng = np.random.default_rng(300 + 10 * variant + seed)
    base = w.batched(seed=15 + seed, scale=0.002).db
    db2, q_sat, _ = w.plant_saturating(base, w.draw_residues(rng, 20), count=2, run=3100)
    lens = [16, 17, 48, 5, 33, 64, 80, 15, 1, 1, 100, 47, 31, 16, 0, 200, 3, 9, 112, 129]
    rng.shuffle(lens)
    qs = [w.draw_residues(rng, n) for n in lens] + [q_sat]
    sm = w.blosum62()
    exp = _oracle_all(qs, db2, sm, 10, 2)
    with sw.sw_db_load(db2.residues, db2.offsets, w.ALPHABET_SIZE, long_cutoff=4096) as h:
        sw.sw_db_set_variant(h, variant)
        got = sw.sw_search_batch(h, qs, sm, 10, 2)
        st = sw.sw_get_stats(h)
        assert st["multi_query"] == 1 and st["flagged"] >= 2
    _check(got, exp, f"short queries, variant {variant}")


@pytest.mark.parametrize("split", ["0", "1", "3", "auto"])
def test_group_routing_to_intra_kernel(sw, split, monkeypatch):
    """Groups above the split run on the int32 intra-task kernel (one warp per pair); the
    scores do not depend on where the split falls (single- and multi-query batches)."""
    if split != "auto":
        monkeypatch.setenv("SWGB_GROUP_SPLIT", split)
    wl = w.plain(seed=31, scale=0.03)                # ~300 sequences = 5 groups
    rng = np.random.default_rng(7)
    qs1 = [wl.queries[0]]
    qs2 = [wl.queries[0], w.draw_residues(rng, 77), w.draw_residues(rng, 300)]
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        got1 = sw.sw_search_batch(h, qs1, wl.matrix, 10, 2)
        st1 = sw.sw_get_stats(h)
        got2 = sw.sw_search_batch(h, qs2, wl.matrix, 10, 2)
    _check(got1, _oracle_all(qs1, wl.db, wl.matrix, 10, 2), f"split {split} single")
    _check(got2, _oracle_all(qs2, wl.db, wl.matrix, 10, 2), f"split {split} multi")
    if split in ("0", "auto"):
        assert st1["intra_ms"] > 0      # a small database routes its long groups


def test_concurrent_searches_on_one_handle(sw):
    """Four host threads search one database handle at once (calls are serialised inside the
    library; plans and graphs are shared): every result equals the sequential one."""
    import threading
    wl = w.plain(seed=41, scale=0.05)
    rng = np.random.default_rng(43)
    qs = [w.draw_residues(rng, int(m)) for m in rng.integers(1, 400, size=16)]
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        ref = [sw.sw_search(h, q, wl.matrix, 10, 2) for q in qs]
        out, errors = [None] * len(qs), []

        def client(ids):
            try:
                for i in ids:
                    out[i] = sw.sw_search(h, qs[i], wl.matrix, 10, 2)
                    if i % 3 == 0:
                        b = sw.sw_search_batch(h, [qs[i], qs[(i + 1) % len(qs)]], wl.matrix, 10, 2)
                        assert np.array_equal(b[0], ref[i]) and np.array_equal(b[1], ref[(i + 1) % len(qs)])
            except Exception as exc:   # surfaced below
                errors.append(exc)

        threads = [threading.Thread(target=client, args=(list(range(c, len(qs), 4)),)) for c in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    assert not errors, errors
    for i in range(len(qs)):
        assert np.array_equal(out[i], ref[i]), f"query {i}"
    _check(np.stack(ref[:2]), _oracle_all(qs[:2], wl.db, wl.matrix, 10, 2), "sequential reference")


def test_very_long_query(sw):
    """A 20,000-residue query (many strips of the inter-task kernel, 40 passes of the int32
    kernel) against short and long subjects, alone and batched with a short query."""
    rng = np.random.default_rng(17)
    lens = np.concatenate([rng.integers(1, 400, size=150), [5000, 9000]])
    db = w.database_from_lengths(rng, lens)
    sm = w.blosum62()
    q = w.draw_residues(rng, 20000)
    q2 = w.draw_residues(rng, 50)
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, long_cutoff=4096) as h:
        got = sw.sw_search_batch(h, [q, q2], sm, 10, 2)
        got1 = sw.sw_search(h, q, sm, 10, 2)
    exp = _oracle_all([q, q2], db, sm, 10, 2)
    _check(got, exp, "20,000-residue query, batched")
    _check(got1[None], exp[:1], "20,000-residue query, alone")


def test_routed_groups_pass_heights(sw, monkeypatch):
    """Every group routed (split 0) to the int32 block kernel: the oracle's scores for query
    lengths around its 160-, 256- and 512-row passes (5, 8 and 16 rows per lane), odd subject
    counts (a part-filled last block item) and empty sequences."""
    monkeypatch.setenv("SWGB_GROUP_SPLIT", "0")
    rng = np.random.default_rng(91)
    lens = np.concatenate([rng.integers(1, 700, size=203), [0, 0, 1, 2, 33]])
    db = w.database_from_lengths(rng, lens)
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        for m in (1, 31, 159, 160, 161, 255, 256, 257, 511, 512, 600):
            q = w.draw_residues(rng, m)
            got = sw.sw_search(h, q, sm, 10, 2)
            st = sw.sw_get_stats(h)
            _check(got[None], _oracle_all([q], db, sm, 10, 2), f"m={m}")
            assert st["inter_cells"] == 0 and st["intra_ms"] > 0
        qs = [w.draw_residues(rng, 90), w.draw_residues(rng, 200)]
        got = sw.sw_search_batch(h, qs, sm, 3, 7)
    _check(got, _oracle_all(qs, db, sm, 3, 7), "batch, gaps 3/7")


@pytest.mark.parametrize("k", [1, 5, 64, 1000, 4096])
def test_sorting_stage_topk(sw, k):
    """Sorting stage: device top-k equals a full sort by (descending score, ascending index)
    of the oracle's scores; heavy ties (random small scores) and large scores (> 2^16, so the
    radix select runs over several digits) included."""
    import torch
    rng = np.random.default_rng(k)
    n = 9000
    rows = [rng.integers(0, 40, size=n), rng.integers(0, 3_000_000, size=n),
            np.zeros(n, np.int64), np.concatenate([np.full(n - 3, 7), [70000, 70000, 9]])]
    sc = np.stack(rows).astype(np.int32)
    d = torch.from_numpy(sc.reshape(-1)).cuda()
    top_s, top_i = sw.sw_topk(d, n, sc.shape[0], k)
    torch.cuda.synchronize()
    for q in range(sc.shape[0]):
        order = np.lexsort((np.arange(n), -sc[q].astype(np.int64)))[:k]
        assert np.array_equal(top_i[q].cpu().numpy(), order), f"row {q}"
        assert np.array_equal(top_s[q].cpu().numpy(), sc[q][order]), f"row {q}"


def test_sorting_stage_after_search(sw):
    """Search then sort on the device: the top hits are the oracle's best scores."""
    import torch
    wl = w.plain(seed=41, scale=0.1)
    db2, q2, planted = w.plant_saturating(wl.db, wl.queries[0], count=4, run=3100)
    with sw.sw_db_load(db2.residues, db2.offsets, w.ALPHABET_SIZE) as h:
        dq = torch.from_numpy(q2).cuda()
        out = torch.empty(h.num_seqs, dtype=torch.int32, device="cuda")
        sw.sw_search_batch_device(h, dq, np.array([0, len(q2)], np.int64), wl.matrix, 10, 2, out)
        top_s, top_i = sw.sw_topk(out, h.num_seqs, 1, 10)
        torch.cuda.synchronize()
    exp = _oracle_all([q2], db2, wl.matrix, 10, 2)[0]
    order = np.lexsort((np.arange(len(exp)), -exp))[:10]
    assert np.array_equal(top_i[0].cpu().numpy(), order)
    assert set(planted) <= set(order.tolist())


def test_host_placement_streams_the_database(sw):
    """SW_PLACE_HOST: the database stays in pinned host memory and the kernels read it over
    the CPU-GPU link; scores are identical (long subjects and routed groups included)."""
    rng = np.random.default_rng(17)
    lens = np.concatenate([rng.integers(0, 400, size=500), rng.integers(3000, 5000, size=4)])
    db = w.database_from_lengths(rng, lens)
    qs = [w.draw_residues(rng, n) for n in (150, 700)]
    sm = w.blosum62()
    exp = _oracle_all(qs, db, sm, 10, 2)
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, placement=sw.PLACE_HOST) as h:
        got = sw.sw_search_batch(h, qs, sm, 10, 2)
        got1 = sw.sw_search(h, qs[0], sm, 10, 2)
    _check(got, exp, "host placement")
    _check(got1[None], exp[:1], "host placement, one query")
