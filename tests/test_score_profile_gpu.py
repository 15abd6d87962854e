"""GPU parity of the score-profile form of the single-query inter-task kernel (Section 4.3's
second way to fetch substitution scores; selected by SWGB_SCORE_PROFILE=1): bit-exact with the
oracle over strip boundaries, alphabet sizes up to 32 letters, asymmetric matrices, gap regimes
of the int16 path and planted hits that saturate int16 lanes."""

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


@pytest.fixture(autouse=True)
def _score_profile(monkeypatch):
    monkeypatch.setenv("SWGB_SCORE_PROFILE", "1")
    monkeypatch.setenv("SWGB_GROUP_SPLIT", "1000000000")   # every group on the inter-task kernel


def _search_one(sw, db, q, sm, A, goe, ge, **kw):
    with sw.sw_db_load(db.residues, db.offsets, A, **kw) as h:
        got = sw.sw_search(h, q, sm, goe, ge)
        st = sw.sw_get_stats(h)
    return np.asarray(got, np.int64), st


def _expect(q, db, sm, goe, ge):
    return oracle.sw_search(q, db.residues, db.offsets, sm, goe, ge)[0]


@pytest.mark.parametrize("m", [1, 2, 31, 32, 33, 64, 65, 130, 257])
def test_query_lengths_around_strips(sw, m):
    rng = np.random.default_rng(100 + m)
    lens = np.concatenate([rng.integers(1, 300, size=190), [0, 1, 7, 8, 9, 16]])
    db = w.database_from_lengths(rng, lens)
    q = w.draw_residues(rng, m)
    sm = w.blosum62()
    got, st = _search_one(sw, db, q, sm, w.ALPHABET_SIZE, 10, 2)
    assert st["score_profile"] == 1
    np.testing.assert_array_equal(got, _expect(q, db, sm, 10, 2))


@pytest.mark.parametrize("A", [1, 4, 20, 31, 32])
def test_alphabets_and_asymmetric_matrices(sw, A):
    rng = np.random.default_rng(200 + A)
    sm = rng.integers(-6, 9, size=(A, A)).astype(np.int8)
    lens = rng.integers(0, 250, size=160)
    offs = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    db = w.Database(rng.integers(0, A, size=int(offs[-1])).astype(np.uint8), offs)
    q = rng.integers(0, A, size=77).astype(np.uint8)
    got, st = _search_one(sw, db, q, sm, A, 7, 3)
    assert st["score_profile"] == 1
    np.testing.assert_array_equal(got, _expect(q, db, sm, 7, 3))


@pytest.mark.parametrize("goe,ge", [(0, 0), (3, 7), (12, 2), (16383, 16383)])
def test_gap_regimes(sw, goe, ge):
    rng = np.random.default_rng(goe + 3 * ge)
    db = w.database_from_lengths(rng, rng.integers(0, 200, size=150))
    q = w.draw_residues(rng, 90)
    sm = w.blosum62()
    got, st = _search_one(sw, db, q, sm, w.ALPHABET_SIZE, goe, ge)
    assert st["score_profile"] == 1
    np.testing.assert_array_equal(got, _expect(q, db, sm, goe, ge))


def test_saturating_hits_rescored(sw):
    wl = w.plain(seed=5, scale=0.03)
    db2, q2, idx = w.plant_saturating(wl.db, wl.queries[0], count=4, run=3200)
    got, st = _search_one(sw, db2, q2, wl.matrix, w.ALPHABET_SIZE, 10, 2, long_cutoff=8192)
    exp = _expect(q2, db2, wl.matrix, 10, 2)
    np.testing.assert_array_equal(got, exp)
    assert st["score_profile"] == 1 and exp[idx].max() > 32767 and st["flagged"] >= 4


def test_same_scores_as_query_profile(sw, monkeypatch):
    wl = w.plain(seed=6, scale=0.1)
    q = wl.queries[0]
    sp, st = _search_one(sw, wl.db, q, wl.matrix, w.ALPHABET_SIZE, 10, 2)
    monkeypatch.setenv("SWGB_SCORE_PROFILE", "0")
    qp, st0 = _search_one(sw, wl.db, q, wl.matrix, w.ALPHABET_SIZE, 10, 2)
    assert st["score_profile"] == 1 and st0["score_profile"] == 0
    np.testing.assert_array_equal(sp, qp)
