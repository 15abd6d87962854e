"""Seeded synthetic inputs: determinism and the shapes of the configured workloads."""

import numpy as np

import workloads as w


def test_deterministic_and_seeded():
    a, b, c = w.plain(seed=0, scale=0.05), w.plain(seed=0, scale=0.05), w.plain(seed=1, scale=0.05)
    assert np.array_equal(a.db.residues, b.db.residues) and np.array_equal(a.db.offsets, b.db.offsets)
    assert not np.array_equal(a.db.offsets, c.db.offsets)
    assert np.array_equal(a.queries[0], b.queries[0])


def test_plain_shape():
    wl = w.plain()
    lens = wl.db.lengths()
    assert wl.db.num_seqs == 10_000 and lens.min() >= 20 and lens.max() <= 2000
    assert 240 < lens.mean() < 260
    assert len(wl.queries) == 1 and len(wl.queries[0]) == 144
    assert wl.db.residues.max() < 20
    assert wl.gap_open == 10 and wl.gap_extend == 2


def test_query_lengths():
    assert w.PAPER_QUERY_LENGTHS[0] == 144 and w.PAPER_QUERY_LENGTHS[-1] == 5478
    assert sum(w.PAPER_QUERY_LENGTHS) == 30747 and len(w.PAPER_QUERY_LENGTHS) == 20
    assert w.LONG_QUERY_LENGTHS == [1000, 1495, 2236, 3344, 5000]


def test_background_composition():
    rng = np.random.default_rng(0)
    r = w.draw_residues(rng, 2_000_000)
    freq = np.bincount(r, minlength=20) / r.size
    assert np.abs(freq - w.BACKGROUND / w.BACKGROUND.sum()).max() < 2e-3


def test_long_subject_shape_small():
    wl = w.long_subject(scale=0.002)
    lens = wl.db.lengths()
    assert lens.min() >= 5000 and lens.max() <= 35000


def test_plant_saturating():
    wl = w.plain(scale=0.01)
    db2, q2, idx = w.plant_saturating(wl.db, wl.queries[0], count=4, run=3200)
    assert db2.num_seqs == wl.db.num_seqs and len(q2) == 144 + 3200
    for k, i in enumerate(idx):
        s = db2.seq(i)
        assert (s == w.CODE_W).sum() >= 3200
