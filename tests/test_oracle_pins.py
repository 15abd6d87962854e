"""Pins for the CPU oracle: things the paper and the mathematics fix, none of them the
oracle's own recurrence retyped.

* brute-force enumeration of every local alignment on inputs of length <= 6
  (the definition Eqs. sw2-sw4 of the paper's Section 2 compute);
* hand-worked examples (tests/golden/hand_examples.tsv);
* closed forms: self-score under a diagonal-dominant matrix, the ungapped limit (Kadane's
  maximum subarray along each diagonal), the linear-gap special case (a one-matrix
  recurrence), a single residue, empty inputs;
* invariants: score >= 0, transposition symmetry, monotone in the gap costs, upper and
  lower bounds, concatenation;
* a mutation battery showing that plausible mistakes planted in a copy of the oracle's
  C source (on the CPU) fail these pins.
"""

import os
import random
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from bruteforce import local_score
from workloads import blosum62, encode

HERE = os.path.dirname(os.path.abspath(__file__))


def score(q, d, sm, goe, ge, lib=None):
    return oracle.sw_score(np.asarray(q, np.uint8), np.asarray(d, np.uint8), sm, goe, ge, lib=lib)


def _rand_case(rng, max_len=6):
    a = rng.randint(2, 4)
    sm = np.array([[rng.randint(-4, 11) for _ in range(a)] for _ in range(a)], dtype=np.int8)
    q = [rng.randrange(a) for _ in range(rng.randint(0, max_len))]
    d = [rng.randrange(a) for _ in range(rng.randint(0, max_len))]
    goe, ge = rng.randint(0, 12), rng.randint(0, 12)
    return q, d, sm, goe, ge


# ----------------------------------------------------------------------------- brute force
def test_bruteforce_random_small():
    rng = random.Random(1702)
    for _ in range(400):
        q, d, sm, goe, ge = _rand_case(rng)
        assert score(q, d, sm, goe, ge) == local_score(q, d, sm, goe, ge), (q, d, sm, goe, ge)


@pytest.mark.parametrize("goe,ge", [(0, 0), (0, 5), (5, 0), (3, 7), (12, 2), (10, 2), (1, 1)])
def test_bruteforce_gap_regimes(goe, ge):
    """Includes goe < ge, zero costs, the paper's literal (12, 2) and the (10, 2) setting."""
    rng = random.Random(goe * 100 + ge)
    for _ in range(40):
        q, d, sm, _, _ = _rand_case(rng)
        assert score(q, d, sm, goe, ge) == local_score(q, d, sm, goe, ge)


def test_bruteforce_blosum62_length6():
    rng = random.Random(7)
    sm = blosum62()
    for _ in range(25):
        q = [rng.randrange(20) for _ in range(6)]
        d = [rng.randrange(20) for _ in range(6)]
        for goe, ge in [(10, 2), (12, 2), (4, 1), (2, 3)]:
            assert score(q, d, sm, goe, ge) == local_score(q, d, sm, goe, ge)


# ----------------------------------------------------------------------------- hand-worked
def _hand_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "hand_examples.tsv")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            q, d, goe, ge, s = ln.rstrip("\n").split("\t")[:5]
            rows.append((q, d, int(goe), int(ge), int(s)))
    return rows


AB = np.array([[3, -3], [-3, 3]], dtype=np.int8)


def _ab(s):
    return [0 if c == "A" else 1 for c in s]


@pytest.mark.parametrize("row", _hand_rows())
def test_hand_worked(row):
    q, d, goe, ge, expect = row
    assert score(_ab(q), _ab(d), AB, goe, ge) == expect
    assert local_score(_ab(q), _ab(d), AB, goe, ge) == expect


# ----------------------------------------------------------------------------- closed forms
def _diag_dominant(sm, letters):
    for a in letters:
        if sm[a, a] <= 0:
            return False
        for b in letters:
            if a != b and 2 * int(sm[a, b]) > int(sm[a, a]) + int(sm[b, b]):
                return False
    return True


def test_blosum62_table_properties():
    sm = blosum62()
    assert sm.shape == (24, 24) and (sm == sm.T).all()
    assert sm.min() == -4 and sm.max() == 11
    assert _diag_dominant(sm, range(20))
    assert int(sm[17, 17]) == 11 and int(sm[4, 4]) == 9  # W/W and C/C


def test_self_score_closed_form():
    """Diagonal-dominant SM with a positive diagonal: score(q, q) = sum_i SM(q_i, q_i)."""
    sm = blosum62()
    rng = np.random.default_rng(3)
    for m in [1, 2, 7, 50, 300, 1000]:
        q = rng.integers(0, 20, size=m).astype(np.uint8)
        expect = int(sum(int(sm[c, c]) for c in q))
        for goe, ge in [(10, 2), (12, 2), (0, 0), (1, 5)]:
            assert score(q, q, sm, goe, ge) == expect


def _kadane_diagonals(q, d, sm):
    best = 0
    m, n = len(q), len(d)
    for off in range(-(m - 1), n):
        run = 0
        for i in range(m):
            j = i + off
            if 0 <= j < n:
                run = max(0, run + int(sm[q[i], d[j]]))
                best = max(best, run)
    return best


def test_ungapped_limit_is_kadane_per_diagonal():
    sm = blosum62()
    rng = np.random.default_rng(4)
    for _ in range(30):
        q = rng.integers(0, 20, size=int(rng.integers(1, 60))).astype(np.uint8)
        d = rng.integers(0, 20, size=int(rng.integers(1, 60))).astype(np.uint8)
        big = 10 ** 6
        assert score(q, d, sm, big, big) == _kadane_diagonals(q, d, sm)


def _linear_gap(q, d, sm, g):
    """Linear gaps (goe == ge == g): a single matrix, H = max(0, diag + s, up - g, left - g)."""
    m, n = len(q), len(d)
    prev = [0] * (n + 1)
    best = 0
    for i in range(1, m + 1):
        cur = [0] * (n + 1)
        for j in range(1, n + 1):
            cur[j] = max(0, prev[j - 1] + int(sm[q[i - 1], d[j - 1]]), prev[j] - g, cur[j - 1] - g)
            best = max(best, cur[j])
        prev = cur
    return best


def test_linear_gap_special_case():
    sm = blosum62()
    rng = np.random.default_rng(5)
    for _ in range(30):
        q = rng.integers(0, 20, size=int(rng.integers(1, 40))).astype(np.uint8)
        d = rng.integers(0, 20, size=int(rng.integers(1, 40))).astype(np.uint8)
        for g in [0, 1, 2, 4, 11]:
            assert score(q, d, sm, g, g) == _linear_gap(q, d, sm, g)


def test_single_residue():
    sm = blosum62()
    rng = np.random.default_rng(6)
    for _ in range(20):
        a = int(rng.integers(0, 24))
        d = rng.integers(0, 24, size=int(rng.integers(1, 50))).astype(np.uint8)
        expect = max(0, max(int(sm[a, x]) for x in d))
        assert score([a], d, sm, 10, 2) == expect
        assert score(d, [a], sm, 10, 2) == max(0, max(int(sm[x, a]) for x in d))


def test_empty_inputs():
    sm = blosum62()
    q = encode("MKTAYIAKQR")
    assert score([], q, sm, 10, 2) == 0
    assert score(q, [], sm, 10, 2) == 0
    assert score([], [], sm, 10, 2) == 0


# ----------------------------------------------------------------------------- invariants
def test_transposition_symmetry_asymmetric_matrix():
    """score(q, d, SM) = score(d, q, SM^T): catches a transposed matrix index."""
    rng = np.random.default_rng(8)
    for _ in range(40):
        a = int(rng.integers(2, 6))
        sm = rng.integers(-4, 12, size=(a, a)).astype(np.int8)
        q = rng.integers(0, a, size=int(rng.integers(1, 30))).astype(np.uint8)
        d = rng.integers(0, a, size=int(rng.integers(1, 30))).astype(np.uint8)
        goe, ge = int(rng.integers(0, 13)), int(rng.integers(0, 13))
        assert score(q, d, sm, goe, ge) == score(d, q, sm.T.copy(), goe, ge)


def test_invariants_blosum62():
    sm = blosum62()
    max_s = int(sm.max())
    rng = np.random.default_rng(9)
    for _ in range(25):
        q = rng.integers(0, 20, size=int(rng.integers(1, 80))).astype(np.uint8)
        d1 = rng.integers(0, 20, size=int(rng.integers(1, 80))).astype(np.uint8)
        d2 = rng.integers(0, 20, size=int(rng.integers(1, 80))).astype(np.uint8)
        s = score(q, d1, sm, 10, 2)
        assert s >= 0
        assert s == score(d1, q, sm, 10, 2)                        # symmetric SM
        assert s <= min(len(q), len(d1)) * max_s
        assert s >= max(0, int(sm[np.ix_(q, d1)].max()))
        cat = np.concatenate([d1, d2])
        assert score(q, cat, sm, 10, 2) >= max(s, score(q, d2, sm, 10, 2))
        prev = None
        for goe in [0, 2, 5, 10, 20]:                              # non-increasing in goe
            v = score(q, d1, sm, goe, 2)
            assert prev is None or v <= prev
            prev = v
        prev = None
        for ge in [0, 1, 2, 5, 10]:                                # non-increasing in ge
            v = score(q, d1, sm, 10, ge)
            assert prev is None or v <= prev
            prev = v


def test_search_equals_pairwise_and_threads():
    sm = blosum62()
    rng = np.random.default_rng(10)
    seqs = [rng.integers(0, 20, size=int(rng.integers(0, 120))).astype(np.uint8) for _ in range(60)]
    offs = np.zeros(61, np.int64)
    np.cumsum([len(s) for s in seqs], out=offs[1:])
    res = np.concatenate(seqs)
    q = rng.integers(0, 20, size=90).astype(np.uint8)
    one, _ = oracle.sw_search(q, res, offs, sm, 10, 2, threads=1)
    many, used = oracle.sw_search(q, res, offs, sm, 10, 2, threads=4)
    expect = [score(q, s, sm, 10, 2) for s in seqs]
    assert one.tolist() == expect and many.tolist() == expect and used >= 1
    pairs = oracle.sw_pairs([q, q[:10]], res, offs, [0, 1, 1], [3, 3, 59], sm, 10, 2)
    assert pairs.tolist() == [expect[3], score(q[:10], seqs[3], sm, 10, 2),
                              score(q[:10], seqs[59], sm, 10, 2)]


# ----------------------------------------------------------------------------- mutations
MUTATIONS = {
    "drop_zero": ("max2(0, Hp[j - 1] + (int64_t)row[s2[j - 1]])",
                  "(Hp[j - 1] + (int64_t)row[s2[j - 1]])"),
    "e_sign": ("Ec[j - 1] - ge", "Ec[j - 1] + ge"),
    "f_uses_goe_for_extend": ("Fp[j] - ge", "Fp[j] - goe"),
    "transposed_matrix": ("row[s2[j - 1]]",
                          "sm[(size_t)s2[j - 1] * (size_t)alphabet + s1[i - 1]]"),
    "diag_off_by_one": ("max2(0, Hp[j - 1] +", "max2(0, Hp[j] +"),
    "drop_e_term": ("h = max2(h, Ec[j]);", ""),
    "drop_f_term": ("h = max2(h, Fc[j]);", ""),
    "skip_last_row": ("for (int64_t i = 1; i <= m; ++i)", "for (int64_t i = 1; i < m; ++i)"),
    "open_from_e": ("Ec[j] = max2(Hc[j - 1] - goe", "Ec[j] = max2(Hc[j - 1] - ge"),
}


def _pins_pass(lib) -> bool:
    rng = random.Random(99)
    for q, d, goe, ge, expect in _hand_rows():
        if score(_ab(q), _ab(d), AB, goe, ge, lib=lib) != expect:
            return False
    for _ in range(150):
        q, d, sm, goe, ge = _rand_case(rng)
        if score(q, d, sm, goe, ge, lib=lib) != local_score(q, d, sm, goe, ge):
            return False
    r2 = np.random.default_rng(8)
    for _ in range(20):
        a = int(r2.integers(2, 6))
        sm = r2.integers(-4, 12, size=(a, a)).astype(np.int8)
        q = r2.integers(0, a, size=int(r2.integers(1, 30))).astype(np.uint8)
        d = r2.integers(0, a, size=int(r2.integers(1, 30))).astype(np.uint8)
        if score(q, d, sm, 3, 1, lib=lib) != score(d, q, sm.T.copy(), 3, 1, lib=lib):
            return False
    return True


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_planted_mistakes_fail_pins(tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "sw_oracle.c")).read()
    assert _pins_pass(oracle.load())
    survivors = []
    for name, (old, new) in MUTATIONS.items():
        assert old in src, f"mutation {name}: pattern not found in oracle source"
        path = tmp_path / f"{name}.c"
        path.write_text(src.replace(old, new, 1))
        so = str(tmp_path / f"lib{name}.so")
        subprocess.run(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-o", so, str(path)],
                       check=True)
        if _pins_pass(oracle.load(so)):
            survivors.append(name)
    assert not survivors, f"planted mistakes not caught by the pins: {survivors}"
