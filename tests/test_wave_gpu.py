"""GPU parity of the packed int16x2 wavefront kernel (two queries per register against one
long subject; the intra-task scheme of Section 1 on Eqs. sw2-sw4) against the oracle,
tolerance 0 (integer scores).

Cases: query lengths around the pass heights of the variants (256, 384 and 512 rows), empty
and one-residue queries, several queries per stream (a half restarts from the zero boundary while
the other continues), many short queries packed several to a pass at lane granularity (queries
shorter than one lane's rows, queries ending and starting inside a pass), subject lengths around the 32-column blocks of the wavefront, gap-cost
regimes, small and asymmetric alphabets, planted hits above the int16 range (flagged and
rescored in int32, with and without overflow of the saturation list), and equality with the
int32 kernels (SWGB_WAVE=0).
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


def _oracle(queries, db, sm, goe, ge):
    return np.stack([oracle.sw_search(q, db.residues, db.offsets, sm, goe, ge)[0] for q in queries])


def _check(got, exp, what):
    got = np.asarray(got, dtype=np.int64)
    bad = np.argwhere(got != exp)
    if bad.size:
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches; first at {i}: gpu {got[i]} oracle {exp[i]}")


def _db(rng, n_short=60, long_lens=(33, 63, 64, 65, 95, 96, 97, 200, 511, 1000, 1500)):
    lens = np.concatenate([rng.integers(0, 30, size=n_short), np.array(long_lens)])
    rng.shuffle(lens)
    return w.database_from_lengths(rng, lens)


@pytest.mark.parametrize("qlens", [
    [256, 100],                       # 8 rows per lane (256-row passes)
    [255, 257, 1, 0, 513],            # empty and one-residue queries, ragged passes
    [1024, 700, 512, 511, 300, 90],   # 16 rows per lane, several queries per stream
    [3000, 40],                       # one long stream against a short one
    [5, 1, 13, 12, 11, 24, 25, 100, 7, 3, 16, 17, 33, 2, 9, 48, 300, 0, 8, 384],   # several per pass
])
@pytest.mark.parametrize("rows", ["8", "12", "16"])
def test_two_query_wavefront_matches_oracle(sw, qlens, rows, monkeypatch):
    """Every pass height (256, 384 and 512 rows)."""
    monkeypatch.setenv("SWGB_WAVE_ROWS", rows)
    rng = np.random.default_rng(sum(qlens))
    db = _db(rng)
    qs = [w.draw_residues(rng, n) for n in qlens]
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, long_cutoff=32) as h:
        got = sw.sw_search_batch(h, qs, sm, 10, 2)
        st = sw.sw_get_stats(h)
    _check(got, _oracle(qs, db, sm, 10, 2), f"query lengths {qlens}")
    assert st["intra_packed"] == 1 and st["intra_ms"] > 0


@pytest.mark.parametrize("goe,ge", [(0, 0), (1, 5), (12, 2), (3, 1), (16383, 16383)])
def test_gap_regimes(sw, goe, ge):
    rng = np.random.default_rng(goe * 31 + ge)
    db = _db(rng)
    qs = [w.draw_residues(rng, n) for n in (300, 77, 520)]
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, long_cutoff=32) as h:
        got = sw.sw_search_batch(h, qs, sm, goe, ge)
        st = sw.sw_get_stats(h)
    _check(got, _oracle(qs, db, sm, goe, ge), f"gaps {goe}/{ge}")
    assert st["intra_packed"] == 1


@pytest.mark.parametrize("A", [1, 2, 5, 32])
def test_alphabets_and_asymmetric_matrix(sw, A):
    rng = np.random.default_rng(100 + A)
    sm = rng.integers(-6, 12, size=(A, A)).astype(np.int8)
    lens = np.concatenate([rng.integers(0, 40, size=30), [70, 129, 640]])
    offs = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    db = w.Database(rng.integers(0, A, size=int(offs[-1])).astype(np.uint8), offs)
    qs = [rng.integers(0, A, size=n).astype(np.uint8) for n in (260, 33, 600)]
    with sw.sw_db_load(db.residues, db.offsets, A, long_cutoff=64) as h:
        got = sw.sw_search_batch(h, qs, sm, 7, 1)
    _check(got, _oracle(qs, db, sm, 7, 1), f"alphabet {A}")


@pytest.mark.parametrize("flag_cap", [0, 1])
def test_saturated_long_subjects_rescored(sw, flag_cap):
    """Long subjects whose best alignment with a query exceeds the int16 range: the packed
    kernel flags them and the int32 rescore gives the exact score; with a one-entry saturation
    list the rescore sweeps every score instead."""
    rng = np.random.default_rng(5)
    run = np.full(3100, w.CODE_W, np.uint8)
    seqs = [w.draw_residues(rng, n) for n in rng.integers(0, 50, size=40)]
    seqs += [np.concatenate([w.draw_residues(rng, 20), run]), run[:3050],
             w.draw_residues(rng, 900), np.concatenate([run[:3000], w.draw_residues(rng, 10)])]
    db = w.from_sequences(seqs)
    q_sat = np.concatenate([w.encode("MKT"), run[:3005]])
    qs = [q_sat, w.draw_residues(rng, 400), q_sat[:2000]]
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, long_cutoff=128,
                       flag_cap=flag_cap) as h:
        got = sw.sw_search_batch(h, qs, sm, 10, 2)
        st = sw.sw_get_stats(h)
    exp = _oracle(qs, db, sm, 10, 2)
    _check(got, exp, f"saturation, flag_cap {flag_cap}")
    assert exp.max() > 32767 and st["flagged"] >= 3 and st["intra_packed"] == 1


def test_equals_int32_kernels(sw, monkeypatch):
    """The same search with the packed kernel and with the int32 kernels (SWGB_WAVE=0)."""
    rng = np.random.default_rng(11)
    lens = np.concatenate([rng.integers(0, 400, size=150), rng.integers(3100, 5000, size=12)])
    db = w.database_from_lengths(rng, lens)
    qs = [w.draw_residues(rng, n) for n in (144, 1434, 807, 5478, 211)]
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        packed = sw.sw_search_batch(h, qs, sm, 10, 2)
        assert sw.sw_get_stats(h)["intra_packed"] == 1
        monkeypatch.setenv("SWGB_WAVE", "0")
        plain32 = sw.sw_search_batch(h, qs, sm, 10, 2)
        assert sw.sw_get_stats(h)["intra_packed"] == 0
    np.testing.assert_array_equal(packed, plain32)
    _check(packed, _oracle(qs, db, sm, 10, 2), "packed vs oracle")


# ------------------------------------------------------------------ two-subject mode
@pytest.mark.parametrize("half", ["0", "1", "300"])
@pytest.mark.parametrize("long_pairs", ["0", "7", "100000"])
@pytest.mark.parametrize("m", [1, 31, 143, 144, 145, 159, 160, 161, 256, 288, 289, 300, 321, 700])
def test_two_subject_wavefront_matches_oracle(sw, m, long_pairs, half, monkeypatch):
    """One query against a small database whose groups are all routed off the inter-task
    kernel: the two subjects of each slot pair share a warp; the longest pairs run first on
    32-lane wavefronts (passes of 160 or 256 rows: none, seven pairs, or all); the rest run on
    32-lane wavefronts (half 0), on two 16-lane wavefronts of 144-row passes per warp (half 1:
    two slot pairs per item, an odd count leaving one wavefront empty), or on 32-lane
    wavefronts up to pair 300 and 16-lane ones after it."""
    monkeypatch.setenv("SWGB_GROUP_SPLIT", "0")
    monkeypatch.setenv("SWGB_LONG_PAIRS", long_pairs)
    if half == "300":
        monkeypatch.setenv("SWGB_PAIR_HALF_FROM", half)
    else:
        monkeypatch.setenv("SWGB_PAIR_HALF", half)
    rng = np.random.default_rng(1000 + m)
    lens = np.concatenate([rng.integers(0, 500, size=200), [0, 1, 31, 32, 33, 1200], rng.integers(0, 9, size=7)])
    db = w.database_from_lengths(rng, lens)          # 213 sequences: the last group has fillers
    q = w.draw_residues(rng, m)
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        got = sw.sw_search(h, q, sm, 10, 2)
        st = sw.sw_get_stats(h)
    _check(got[None], _oracle([q], db, sm, 10, 2), f"m={m}")
    assert st["intra_packed"] == 2 and st["inter_cells"] == 0
    if half == "1":
        assert st["wave_lanes"] == 16
    elif half == "0":
        assert st["wave_lanes"] == 32


@pytest.mark.parametrize("half", ["0", "1"])
@pytest.mark.parametrize("long_pairs", ["0", "100000"])
@pytest.mark.parametrize("goe,ge", [(0, 0), (2, 9), (12, 2), (16383, 1), (16383, 16383)])
def test_two_subject_gap_regimes_and_alphabet(sw, goe, ge, long_pairs, half, monkeypatch):
    """Gap regimes (the first phase unrolls the F recurrence when Goe + rows x min(Ge, Goe)
    fits int16, and keeps the row-by-row chain otherwise), asymmetric matrix, 7 letters, both
    bulk shapes."""
    monkeypatch.setenv("SWGB_GROUP_SPLIT", "0")
    monkeypatch.setenv("SWGB_LONG_PAIRS", long_pairs)
    monkeypatch.setenv("SWGB_PAIR_HALF", half)
    rng = np.random.default_rng(7 * goe + ge)
    A = 7
    sm = rng.integers(-5, 9, size=(A, A)).astype(np.int8)     # asymmetric
    lens = rng.integers(0, 300, size=150)
    offs = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    db = w.Database(rng.integers(0, A, size=int(offs[-1])).astype(np.uint8), offs)
    q = rng.integers(0, A, size=190).astype(np.uint8)
    with sw.sw_db_load(db.residues, db.offsets, A) as h:
        got = sw.sw_search(h, q, sm, goe, ge)
    _check(got[None], _oracle([q], db, sm, goe, ge), f"gaps {goe}/{ge}")


@pytest.mark.parametrize("half", ["0", "1"])
@pytest.mark.parametrize("flag_cap", [0, 1])
def test_two_subject_saturation_rescored(sw, flag_cap, half, monkeypatch):
    """Hits above the int16 range in the two-subject mode: a matrix whose W/W entry is 120 lets
    a 300-residue query (whose profile fits in shared memory) score 36,000 against a run of W;
    those lanes are flagged and rescored in int32, with and without overflow of the list.  (No
    first phase: the planted subjects are among the longest, which it would align in int32.)"""
    monkeypatch.setenv("SWGB_GROUP_SPLIT", "0")
    monkeypatch.setenv("SWGB_LONG_PAIRS", "0")
    monkeypatch.setenv("SWGB_PAIR_HALF", half)
    wl = w.plain(seed=41, scale=0.03)
    sm = wl.matrix.copy()
    sm[w.CODE_W, w.CODE_W] = 120
    q = np.concatenate([w.draw_residues(np.random.default_rng(2), 20), np.full(300, w.CODE_W, np.uint8)])
    db2, _, idx = w.plant_saturating(wl.db, q[:20], count=5, run=300)
    with sw.sw_db_load(db2.residues, db2.offsets, w.ALPHABET_SIZE, flag_cap=flag_cap) as h:
        got = sw.sw_search(h, q, sm, 10, 2)
        st = sw.sw_get_stats(h)
    exp = _oracle([q], db2, sm, 10, 2)
    _check(got[None], exp, f"saturation, flag_cap {flag_cap}")
    assert exp.max() > 32767 and st["flagged"] >= 3 and st["intra_packed"] == 2


@pytest.mark.parametrize("long_pairs", ["0", "500"])
@pytest.mark.parametrize("m", [1, 33, 144, 160, 250])
def test_two_subject_many_pairs_per_warp(sw, m, long_pairs, monkeypatch):
    """A one-pass query (160 rows, or 256 for m = 250) against 24,000 subjects: about ten slot
    pairs per warp from the work queue, with and without a first phase.  Lengths mix empty
    subjects, very short ones, the bulk of the length law and a few long ones."""
    monkeypatch.setenv("SWGB_GROUP_SPLIT", "0")
    monkeypatch.setenv("SWGB_LONG_PAIRS", long_pairs)
    monkeypatch.setenv("SWGB_PAIR_HALF", "0")
    rng = np.random.default_rng(77 + m)
    n = 24000
    lens = np.where(rng.random(n) < 0.3, rng.integers(0, 40, size=n),
                    np.clip(rng.lognormal(4.3, 0.6, size=n), 1, 1500).astype(np.int64))
    lens[rng.integers(0, n, size=40)] = rng.integers(600, 1500, size=40)
    db = w.database_from_lengths(rng, lens)
    q = w.draw_residues(rng, m)
    sm = w.blosum62()
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        got = sw.sw_search(h, q, sm, 10, 2)
        st = sw.sw_get_stats(h)
    _check(got[None], _oracle([q], db, sm, 10, 2), f"many pairs per warp, m={m}")
    assert st["intra_packed"] == 2 and st["inter_cells"] == 0 and st["wave_lanes"] == 32


def test_two_subject_equals_int32_kernel(sw, monkeypatch):
    wl = w.plain(seed=3, scale=0.3)
    with sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE) as h:
        packed = sw.sw_search(h, wl.queries[0], wl.matrix, 10, 2)
        assert sw.sw_get_stats(h)["intra_packed"] == 2
        monkeypatch.setenv("SWGB_PAIR", "0")
        plain32 = sw.sw_search(h, wl.queries[0], wl.matrix, 10, 2)
        assert sw.sw_get_stats(h)["intra_packed"] == 0
    np.testing.assert_array_equal(packed, plain32)
    _check(packed[None], _oracle(wl.queries, wl.db, wl.matrix, 10, 2), "plain 3,000 sequences")
