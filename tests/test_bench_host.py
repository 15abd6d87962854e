"""Host-side checks of the benchmark's parity and baseline logic (no GPU).

The bench line's `parity` fields come from these checkers, so each is shown to report a score
that differs from the oracle's: the plain configuration's full recomputation, the sampled
check of the larger configurations (which always includes every query's top hit), and the row
hashes of the headline configuration, whose stored oracle results must still match the inputs
the workload generator makes.
"""

import numpy as np
import pytest

import bench
import oracle
import workloads as w


def _oracle_rows(wl):
    return np.stack([oracle.sw_search(q, wl.db.residues, wl.db.offsets, wl.matrix, wl.gap_open,
                                      wl.gap_extend)[0] for q in wl.queries]).astype(np.int32)


def test_plain_parity_reports_a_planted_error():
    wl = w.plain(seed=0, scale=0.02)
    got = _oracle_rows(wl)
    par = bench.parity("plain", wl, got)
    assert par["ok"] and par["scores_checked"] == got.size and par["mismatches"] == 0
    got[0, 17] += 1
    par = bench.parity("plain", wl, got)
    assert not par["ok"] and par["mismatches"] == 1
    cb = bench.config_cpu_baseline("plain", wl, par)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1


def test_sampled_parity_covers_every_top_hit():
    wl = bench.make_workload("long_subject", 0, 0.002)   # 100 subjects: no stored results match
    assert bench.load_golden("long_subject", wl) is None
    got = _oracle_rows(wl)
    par = bench.parity("long_subject", wl, got)
    assert par["ok"] and par["scores_checked"] >= len(wl.queries)
    q = len(wl.queries) - 1
    got[q, int(np.argmax(got[q]))] += 5                  # a wrong top hit of the last query
    par = bench.parity("long_subject", wl, got)
    assert not par["ok"] and par["mismatches"]


def test_row_hash_checker_locates_a_planted_error():
    wl = w.plain(seed=1, scale=0.02)
    got = _oracle_rows(wl)
    blk = 64
    doc = {"block": blk, "rows": [{"sha256": bench.sha(np.ascontiguousarray(r, "<i4")),
                                   "blocks": [bench.sha(np.ascontiguousarray(r[b:b + blk], "<i4"))[:16]
                                              for b in range(0, r.size, blk)]} for r in got]}
    assert bench.check_rows_golden(got, doc)["ok"]
    got[0, 3 * blk + 5] -= 1
    res = bench.check_rows_golden(got, doc)
    assert not res["ok"] and res["bad_rows"] == [0] and res["bad_blocks"] == 1


@pytest.mark.timeout(600)
def test_stored_headline_results_match_the_generated_inputs():
    """The stored oracle row hashes of the 20 x 1M headline search were made from exactly the
    inputs the generator makes now (queries, residues, offsets), so the bench can check every
    score against them."""
    wl = bench.make_workload("batched", 0, 1.0)
    doc = bench.load_golden("batched", wl)
    assert doc is not None and len(doc["rows"]) == len(wl.queries) == 20


@pytest.mark.parametrize("kernel,workload", [("k_inter_mq_i16x2", "batched"),
                                             ("k_inter_mq_i16x2", "paper_shaped"),
                                             ("k_wave_mq_i16x2", "long_subject"),
                                             ("k_wave_ss_i16x2", "plain")])
def test_profiles_of_the_reported_kernels_are_current(kernel, workload):
    """The ncu summary the bench reads for each configuration's dominant kernel was taken on
    the kernel source as it is now (else the bench reports its traffic as unknown)."""
    rows = {"batched": 64, "paper_shaped": 32}.get(workload)
    traffic = bench.ncu_traffic(workload, kernel, rows_per_strip=rows)
    assert traffic is not None and traffic > 0
