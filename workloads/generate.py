"""Seeded synthetic protein workloads shaped like the paper's benchmark (Section 5.1).

The paper searches 20 Swiss-Prot queries (lengths 144..5478) against Environmental NR
(6,962,291 sequences, 1.38G residues).  Neither data set is available, so every workload
here is synthetic: residues are i.i.d. draws from the Robinson & Robinson (1991) amino-acid
background frequencies (the set BLAST uses for BLOSUM62 statistics), sequence lengths follow
``clip(round(lognormal(mu, sigma)), lo, hi)`` with ``mu = ln(mean) - sigma**2 / 2``.

This module holds input generation only; it computes nothing of the alignment method.
Both the CUDA path and the oracle consume what it produces.  Every draw goes through
``numpy.random.default_rng`` (PCG64), which gives identical streams on x86 and Arm.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from .blosum62 import ALPHABET, blosum62

# Robinson & Robinson (1991) background frequencies, BLOSUM62 letter order A R N D C Q E G H I
# L K M F P S T W Y V.
BACKGROUND = np.array(
    [0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295, 0.07377, 0.02199, 0.05142,
     0.09019, 0.05744, 0.02243, 0.03856, 0.05203, 0.07120, 0.05841, 0.01330, 0.03216, 0.06441],
    dtype=np.float64,
)

ALPHABET_SIZE = len(ALPHABET)  # 24 codes; residues are drawn from the first 20
CODE_W = ALPHABET.index("W")   # highest self-score in BLOSUM62 (11)

# The 20 query lengths of the paper's benchmark span 144..5478 (Section 5.1); the synthetic
# stand-in spaces 20 lengths log-uniformly over that range.
PAPER_QUERY_LENGTHS = [int(round(144 * (5478 / 144) ** (k / 19))) for k in range(20)]
LONG_QUERY_LENGTHS = [int(round(1000 * 5 ** (k / 4))) for k in range(5)]

_CHUNK = 1 << 26


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(tag)]))


def _letter_lut() -> np.ndarray:
    """65536-entry inverse-CDF table: a uniform 16-bit draw -> residue code (0..19)."""
    p = BACKGROUND / BACKGROUND.sum()
    edges = np.cumsum(p) * 65536.0
    lut = np.searchsorted(edges, np.arange(65536, dtype=np.float64) + 0.5, side="right")
    return np.minimum(lut, 19).astype(np.uint8)


_LUT = _letter_lut()


def draw_residues(rng: np.random.Generator, count: int) -> np.ndarray:
    """``count`` i.i.d. residue codes from the background distribution (uint8)."""
    out = np.empty(int(count), dtype=np.uint8)
    for lo in range(0, int(count), _CHUNK):
        hi = min(int(count), lo + _CHUNK)
        u = rng.integers(0, 65536, size=hi - lo, dtype=np.uint16)
        np.take(_LUT, u, out=out[lo:hi])
    return out


def lognormal_lengths(rng, n, mean, sigma, lo, hi) -> np.ndarray:
    mu = math.log(mean) - sigma * sigma / 2.0
    x = rng.lognormal(mu, sigma, size=int(n))
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


@dataclasses.dataclass
class Database:
    residues: np.ndarray  # uint8 [R]
    offsets: np.ndarray   # int64 [N+1]

    @property
    def num_seqs(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def num_residues(self) -> int:
        return int(self.offsets[-1])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def seq(self, k: int) -> np.ndarray:
        return self.residues[self.offsets[k]:self.offsets[k + 1]]

    def subset(self, idx) -> "Database":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths()[idx]
        offs = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(lens, out=offs[1:])
        res = np.empty(int(offs[-1]), dtype=np.uint8)
        for t, k in enumerate(idx):
            res[offs[t]:offs[t + 1]] = self.seq(int(k))
        return Database(res, offs)


def database_from_lengths(rng, lengths) -> Database:
    lengths = np.asarray(lengths, dtype=np.int64)
    offs = np.zeros(lengths.shape[0] + 1, dtype=np.int64)
    np.cumsum(lengths, out=offs[1:])
    return Database(draw_residues(rng, int(offs[-1])), offs)


def make_database(num_seqs, mean=250.0, sigma=0.8, lo=20, hi=2000, seed=0,
                  uniform=None) -> Database:
    """Synthetic database: log-normal lengths (or ``uniform=(lo, hi)``), i.i.d. residues."""
    rng_len = _rng(seed, 1)
    if uniform is not None:
        lengths = rng_len.integers(uniform[0], uniform[1] + 1, size=int(num_seqs)).astype(np.int64)
    else:
        lengths = lognormal_lengths(rng_len, num_seqs, mean, sigma, lo, hi)
    return database_from_lengths(_rng(seed, 2), lengths)


def make_queries(lengths, seed=0) -> list:
    rng = _rng(seed, 3)
    return [draw_residues(rng, int(m)) for m in lengths]


@dataclasses.dataclass
class Workload:
    name: str
    queries: list
    db: Database
    matrix: np.ndarray
    gap_open: int = 10   # a gap of length k costs gap_open + (k - 1) * gap_extend
    gap_extend: int = 2

    @property
    def cells(self) -> int:
        return int(sum(len(q) for q in self.queries)) * self.db.num_residues


# Configurations.  ``scale`` shrinks the database (number of sequences) for parity tests.
def plain(seed=0, scale=1.0, query_lengths=None) -> Workload:
    """One 144-residue query vs 10,000 sequences (log-normal mean 250, clip 20..2000)."""
    db = make_database(max(1, int(10_000 * scale)), 250.0, 0.8, 20, 2000, seed=seed)
    ql = [144] if query_lengths is None else query_lengths
    return Workload("plain", make_queries(ql, seed), db, blosum62())


def batched(seed=0, scale=1.0, query_lengths=None) -> Workload:
    """The 20 paper-shaped query lengths vs 1M sequences (log-normal mean 250, clip 20..2000)."""
    db = make_database(max(1, int(1_000_000 * scale)), 250.0, 0.8, 20, 2000, seed=seed)
    ql = PAPER_QUERY_LENGTHS if query_lengths is None else query_lengths
    return Workload("batched", make_queries(ql, seed), db, blosum62())


def paper_shaped(seed=0, scale=1.0, query_lengths=None) -> Workload:
    """The 20 query lengths vs 6M sequences (log-normal mean 250, sigma 1.0, clip 20..35000)."""
    db = make_database(max(1, int(6_000_000 * scale)), 250.0, 1.0, 20, 35000, seed=seed)
    ql = PAPER_QUERY_LENGTHS if query_lengths is None else query_lengths
    return Workload("paper_shaped", make_queries(ql, seed), db, blosum62())


def long_subject(seed=0, scale=1.0, query_lengths=None) -> Workload:
    """Five 1,000..5,000-residue queries vs 50,000 sequences uniform over 5,000..35,000."""
    db = make_database(max(1, int(50_000 * scale)), seed=seed, uniform=(5000, 35000))
    ql = LONG_QUERY_LENGTHS if query_lengths is None else query_lengths
    return Workload("long_subject", make_queries(ql, seed), db, blosum62())


def serving_queries(num, seed=0, mean=400.0, sigma=0.8, lo=50, hi=5000) -> list:
    """Query stream for the serving workload: log-normal lengths (mean 400, clip 50..5000)."""
    lengths = lognormal_lengths(_rng(seed, 4), num, mean, sigma, lo, hi)
    return make_queries(lengths, seed + 7919)


def poisson_arrivals(num, rate_per_s, seed=0) -> np.ndarray:
    """Arrival times (seconds, ascending) of a Poisson process with the given rate."""
    gaps = _rng(seed, 5).exponential(1.0 / float(rate_per_s), size=int(num))
    return np.cumsum(gaps)


def plant_saturating(db: Database, query: np.ndarray, count=4, run=3200, seed=0):
    """Return (db', query') with hits whose score exceeds the int16 range.

    ``query'`` is ``query`` with a run of ``run`` W residues appended; ``count`` database
    sequences (chosen by the seed) are replaced by: copies of ``query'`` and pure W runs.
    BLOSUM62 scores W/W = 11, so a run of 3200 aligned W's scores 35200 > 32767.
    """
    rng = _rng(seed, 6)
    q2 = np.concatenate([query, np.full(run, CODE_W, dtype=np.uint8)])
    idx = set(rng.choice(db.num_seqs, size=min(count, db.num_seqs), replace=False).tolist())
    seqs, k = [], 0
    for i in range(db.num_seqs):
        if i in idx:
            seqs.append(q2.copy() if k % 2 == 0 else np.full(run + k, CODE_W, dtype=np.uint8))
            k += 1
        else:
            seqs.append(db.seq(i))
    return from_sequences(seqs), q2, sorted(idx)


def from_sequences(seqs) -> Database:
    lens = np.array([len(s) for s in seqs], dtype=np.int64)
    offs = np.zeros(len(seqs) + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    res = np.concatenate([np.asarray(s, dtype=np.uint8) for s in seqs]) if seqs else \
        np.zeros(0, dtype=np.uint8)
    return Database(res, offs)


def sample_indices(num_seqs, count, seed=0) -> np.ndarray:
    """A fixed seeded sample of database indices (sorted)."""
    count = min(int(count), int(num_seqs))
    return np.sort(_rng(seed, 8).choice(int(num_seqs), size=count, replace=False))
