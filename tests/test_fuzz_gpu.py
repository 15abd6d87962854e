"""Seeded fuzzing of the whole CUDA path against the oracle (tolerance 0): random alphabet
sizes (1..32), random (also asymmetric) matrices, gap costs across the int16 and int32 paths,
length mixes with empty and one-residue sequences, long-subject cutoffs, kernel variants,
routing splits and saturation-list capacities.  Each case is small enough for the oracle to
check every score."""

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


def _case(seed):
    rng = np.random.default_rng(seed)
    A = int(rng.choice([1, 2, 4, 20, 24, 32]))
    lo, hi = sorted(rng.integers(-12, 16, size=2))
    sm = rng.integers(lo, hi + 1, size=(A, A)).astype(np.int8)
    if rng.random() < 0.3:
        sm = ((sm.astype(np.int16) + sm.T) // 2).astype(np.int8)
    n_seq = int(rng.integers(1, 400))
    kind = rng.integers(3)
    if kind == 0:
        lens = rng.integers(0, 300, size=n_seq)
    elif kind == 1:
        lens = np.clip(rng.lognormal(4.5, 1.0, size=n_seq), 0, 3000).astype(np.int64)
    else:
        lens = rng.choice([0, 1, 2, 7, 8, 9, 63, 64, 65, 1000], size=n_seq)
    offs = np.zeros(n_seq + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    db = w.Database(rng.integers(0, A, size=int(offs[-1])).astype(np.uint8), offs)
    nq = int(rng.integers(1, 6))
    qs = [rng.integers(0, A, size=int(rng.integers(0, 700))).astype(np.uint8) for _ in range(nq)]
    goe = int(rng.choice([0, 1, 3, 10, 12, 40, 20000]))
    ge = int(rng.choice([0, 1, 2, 5, 13]))
    cutoff = int(rng.choice([8, 64, 256, 3072]))
    variant = int(rng.integers(4))
    split = str(int(rng.choice([-1, 0, 1, 2, 1000000])))
    flag_cap = int(rng.choice([0, 0, 1, 3]))
    return A, sm, db, qs, goe, ge, cutoff, variant, split, flag_cap


@pytest.mark.parametrize("seed", list(range(48)))
def test_fuzz_against_oracle(sw, seed, monkeypatch):
    """The batch search, the single-query search of the first query and the no-allocation
    search of the first query; every third seed with the score-profile single-query kernel."""
    import torch
    A, sm, db, qs, goe, ge, cutoff, variant, split, flag_cap = _case(1000 + seed)
    if split != "-1":
        monkeypatch.setenv("SWGB_GROUP_SPLIT", split)
    if seed % 3 == 0:
        monkeypatch.setenv("SWGB_SCORE_PROFILE", "1")
    max_s = max(0, int(sm.max()))
    if max_s * max([len(q) for q in qs] + [1]) > 2**31 - 1:
        pytest.skip("score bound above int32")
    with sw.sw_db_load(db.residues, db.offsets, A, long_cutoff=cutoff, flag_cap=flag_cap) as h:
        sw.sw_db_set_variant(h, variant)
        got = sw.sw_search_batch(h, qs, sm, goe, ge)
        got1 = sw.sw_search(h, qs[0], sm, goe, ge)
        got_na = None
        if len(qs[0]) <= 8192:                   # SW_NOALLOC_MAX_QUERY
            d_q = torch.from_numpy(qs[0]).cuda()
            d_s = torch.full((h.num_seqs,), -9, dtype=torch.int32, device="cuda")
            sw.sw_search_noalloc(h, d_q, sm, goe, ge, d_s)
            got_na = d_s.cpu().numpy()
    what = f"A={A}, goe={goe}, ge={ge}, cutoff={cutoff}, variant={variant}, split={split}"
    for k, q in enumerate(qs):
        exp, _ = oracle.sw_search(q, db.residues, db.offsets, sm, goe, ge)
        bad = np.nonzero(got[k].astype(np.int64) != exp)[0]
        assert bad.size == 0, (f"seed {seed} query {k} (m={len(q)}, {what}): "
                               f"{bad.size} mismatches, first {bad[0]}: {got[k][bad[0]]} vs {exp[bad[0]]}")
        if k == 0:
            np.testing.assert_array_equal(got1.astype(np.int64), exp, err_msg=f"seed {seed} alone, {what}")
            if got_na is not None:
                np.testing.assert_array_equal(got_na.astype(np.int64), exp,
                                              err_msg=f"seed {seed} no-allocation search, {what}")
