"""Benchmark: GCUPS of the Smith-Waterman database search on GB300.

One step = one pass of the whole search (query profiles, inter-task int16x2 kernel,
intra-task kernel for long subjects, int32 rescore of saturated lanes) for a batch of
queries against the device-resident database.  Headline workload: the 20 paper-shaped query
lengths (144..5478, sum 30,747) against a seeded synthetic database of 1M protein
sequences (log-normal lengths, mean 250, clipped to 20..2000; ~249M residues), BLOSUM62,
a gap of length k costing 10 + 2(k - 1).  GCUPS = sum(|Q|) * |D| / (t * 1e9) (paper
Eq. gcups).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  On one GPU the default run also measures, after the
headline, the other workloads -- serving under Poisson arrivals (capacity, p50/p99 latency,
sustained GCUPS at three arrival rates), the plain one-query search, the long-subject mix and
the paper-shaped 6M-sequence search -- each with its GCUPS, the roofline fraction of its
dominant kernel, an end-to-end figure through the C ABI with host buffers and a check against
the oracle; they go under "configs" in the same line (--headline-only skips them).  Under
torchrun each rank searches its own database of the headline size (weak scaling; no
collective on the data path) and only the headline runs.
"""

from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402

# ALU-pipe roofline of the inter-task kernels: the DPX max-plus operations issue on the ALU
# pipe at 64 lane-operations per clock per SM (ncu: the pipe is 92-94% busy; a wall-clock
# rate measurement gave 19.9e12 viaddmax_s16x2 per second at 2,070 MHz on 152 SMs), two cells
# per int16x2 lane-operation, and at least 5.5 ALU operations per cell pair for Eqs. sw2-sw4
# (5 DPX updates + half a three-way max for the running best).
LANE_OPS_PER_CLK_SM = 64
OPS_PER_CELL_PAIR = 5.5
# int32 update: 4 viaddmax + half a vimax3 per cell on the ALU pipe; the subtraction of Goe is a
# plain integer add, which issues on the FMA pipe
ALU_OPS_PER_CELL_I32 = 4.5
CSRC = os.path.join(ROOT, "paper_1702_07195_gb300", "csrc")
GOLDEN = os.path.join(ROOT, "tests", "golden")
# fixed seeded sample of database sequences timed by the oracle (both arms): 1 % of the database
CPU_SAMPLE_FRACTION = 0.01
CPU_SAMPLE_SEED = 1702


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "plain", "paper_shaped", "long_subject", "serving"])
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the other workloads after the headline")
    ap.add_argument("--extra", default="serving,plain,long_subject,paper_shaped",
                    help="workloads measured after the headline (one GPU only)")
    ap.add_argument("--requests", type=int, default=100, help="serving: requests per rate")
    ap.add_argument("--slices", type=int, default=0,
                    help="serving: database slices per scan cycle (0: automatic)")
    ap.add_argument("--rates", default="0.25,0.5,0.9",
                    help="serving: arrival rates as fractions of the measured capacity")
    ap.add_argument("--scale", type=float, default=1.0, help="database scale (tests only)")
    ap.add_argument("--query-lengths", default="",
                    help="comma-separated query lengths replacing the workload's (profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="skip the kernel-variant autotuner")
    ap.add_argument("--variant", type=int, default=-1,
                    help="force an inter-task kernel variant instead of autotuning (profiling)")
    ap.add_argument("--long-cutoff", type=int, default=0,
                    help="subjects longer than this go to the intra-task kernel (0: default)")
    ap.add_argument("--placement", default="device", choices=["device", "host"],
                    help="database in HBM (default) or streamed from pinned host memory")
    ap.add_argument("--score-profile", action="store_true",
                    help="also time the one-query-per-launch pass with the score-profile kernel")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the one-query-per-launch comparison")
    return ap.parse_args()


WORKLOAD_TEXT = {
    "batched": "20 queries (lengths 144..5478 log-uniform, sum 30,747) vs 1M synthetic protein "
               "sequences (log-normal lengths mean 250, clip 20..2000), BLOSUM62, gaps 10/2",
    "plain": "1 query of 144 vs 10,000 synthetic protein sequences (log-normal mean 250, clip "
             "20..2000), BLOSUM62, gaps 10/2",
    "paper_shaped": "20 queries (144..5478) vs 6M synthetic sequences (log-normal mean 250, "
                    "sigma 1.0, clip 20..35,000), BLOSUM62, gaps 10/2",
    "long_subject": "5 queries (1,000..5,000) vs 50,000 synthetic sequences uniform over "
                    "5,000..35,000, BLOSUM62, gaps 10/2",
    "serving": "Poisson arrivals of queries (log-normal lengths mean 400, clip 50..5,000) vs the "
               "resident 1M-sequence synthetic database (batched config), BLOSUM62, gaps 10/2",
}

# Steps of the workloads measured after the headline: (warm-up, timed, end-to-end timed).
EXTRA_STEPS = {"plain": (10, 400, 50), "long_subject": (3, 3, 2), "paper_shaped": (3, 2, 1)}


def make_workload(name, seed, scale, query_lengths=""):
    if name == "serving":
        name = "batched"
    if query_lengths:
        ql = [int(x) for x in query_lengths.split(",") if x]
        return getattr(w, name)(seed=seed, scale=scale, query_lengths=ql)
    return getattr(w, name)(seed=seed, scale=scale)


def workload_config(name, wl):
    """The workload's identity: the same in both arms (ours and the oracle reference)."""
    return {"workload": WORKLOAD_TEXT[name], "queries": len(wl.queries),
            "query_residues": int(sum(len(q) for q in wl.queries)), "db_seqs": wl.db.num_seqs,
            "db_residues": wl.db.num_residues,
            "l2": f"inputs larger than L2 (database {wl.db.num_residues / 1e6:.0f} MB of residues "
                  "resident in HBM and read once per query strip per step)"}


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) taken only while started; start/stop may repeat, and the
    summary covers every sample taken."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.ok = True

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            proc = self.proc
            threading.Thread(target=self._read, args=(proc,), daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None
            self.ok = False

    def _read(self, proc):
        for ln in proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.proc = None

    def summary(self, lines=None) -> dict:
        if not self.ok:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in (self.lines if lines is None else lines):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


class Timed:
    """Context: clock samples during one timed region (kept for the whole-run record too)."""

    def __init__(self, sampler):
        self.s = sampler

    def __enter__(self):
        self.first = len(self.s.lines)
        self.s.start()
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        self.s.stop()
        self.clocks = self.s.summary(self.s.lines[self.first:])


# ---------------------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


KERNEL_SRC = {"k_inter_i16x2": os.path.join(CSRC, "k_inter.cu"),
              "k_inter_mq_i16x2": os.path.join(CSRC, "k_inter_mq.cu"),
              "k_intra_block_i32": os.path.join(CSRC, "k_intra_block.cu"),
              "k_wave_mq_i16x2": os.path.join(CSRC, "k_wave.cu"),
              "k_wave_ss_i16x2": os.path.join(CSRC, "k_wave.cu")}

# rows per strip of the inter-task kernel variants (both kernels), as in csrc/k_inter*.cu
INTER_VARIANT_ROWS = (32, 64, 32, 64)


def ncu_traffic(workload, kernel, rows_per_strip=None):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None
    if the summary is absent, was taken on a different kernel source, or (for the inter-task
    kernels, whose boundary traffic scales with the strip count) on another strip height."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path) or kernel not in KERNEL_SRC:
        return None
    text = open(path).read()
    src = hashlib.sha256(open(KERNEL_SRC[kernel], "rb").read()).hexdigest()[:16]
    m_src = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_src or not m_b or m_src.group(1) != src:
        return None
    m_rows = re.search(r"rows_per_strip:\s*(\d+)", text)
    if m_rows and rows_per_strip is not None and int(m_rows.group(1)) != rows_per_strip:
        return None
    return float(m_b.group(1))


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def load_golden(name, wl):
    """Stored oracle results of a full-size workload (tests/golden/fullsize_<name>.json, written
    by the oracle alone), or None if absent or made from other inputs."""
    path = os.path.join(GOLDEN, f"fullsize_{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        doc = json.load(f)
    fp = doc["inputs"]
    if (fp["num_seqs"] != wl.db.num_seqs or fp["num_residues"] != wl.db.num_residues
            or fp["query_lengths"] != [len(q) for q in wl.queries]
            or fp["queries"] != [sha(q) for q in wl.queries]
            or fp["residues"] != sha(wl.db.residues)):
        return None
    return doc


# ---------------------------------------------------------------------------- oracle baseline
def cpu_sample(wl):
    """The fixed seeded sample of database sequences the oracle is timed on (1 %)."""
    n = wl.db.num_seqs
    count = max(16, int(round(n * CPU_SAMPLE_FRACTION)))
    idx = w.sample_indices(n, count, seed=CPU_SAMPLE_SEED)
    return idx, wl.db.subset(idx)


def host_cores() -> int:
    """Host cores this process may run on (a launcher such as torchrun sets OMP_NUM_THREADS=1
    for its workers, so the oracle is given the count explicitly)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(wl, sub):
    """Times the oracle (as it stands, all host cores) on every query against `sub`."""
    import oracle
    oracle.build()
    cores, threads = 0, host_cores()
    t0 = time.perf_counter()
    for q in wl.queries:
        _, cores = oracle.sw_search(q, sub.residues, sub.offsets, wl.matrix, wl.gap_open,
                                    wl.gap_extend, threads=threads)
    return time.perf_counter() - t0, int(cores)


def sample_text(wl, idx, sub):
    return (f"all {len(wl.queries)} queries vs the fixed seeded 1% sample of the database "
            f"(seed {CPU_SAMPLE_SEED}: {len(idx)} of {wl.db.num_seqs} sequences, "
            f"{sub.num_residues} residues, "
            f"{sum(len(q) for q in wl.queries) * sub.num_residues:.3e} cells)")


def cpu_baseline(wl):
    idx, sub = cpu_sample(wl)
    dt, cores = time_oracle(wl, sub)
    cells = sum(len(q) for q in wl.queries) * sub.num_residues
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": sample_text(wl, idx, sub) + f", timed in {dt:.1f} s"}


def run_reference(args, world, rank):
    """The oracle as the reference arm: the same workload, metric and fixed 1 % sample as our
    arm's cpu_baseline.  The sample is cut into `steps` slices of consecutive sequences; each
    timed step runs every query against one slice, so the timed steps together cover the whole
    sample once.  Warm-up steps run the first slices."""
    if rank != 0:
        return
    wl = make_workload(args.workload, args.seed, args.scale, args.query_lengths)
    idx, sub = cpu_sample(wl)
    k = max(1, args.steps)
    bounds = np.linspace(0, len(idx), k + 1).astype(np.int64)
    slices = [wl.db.subset(idx[bounds[i]:bounds[i + 1]]) for i in range(k)]
    for i in range(args.warmup):
        time_oracle(wl, slices[i % k])
    total, cores = 0.0, 0
    for s in slices:
        dt, cores = time_oracle(wl, s)
        total += dt
    total_m = sum(len(q) for q in wl.queries)
    cells = total_m * sub.num_residues
    value = cells / total / 1e9
    line = {"impl": "reference", "metric": "GCUPS", "value": value, "unit": "GCUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total / k, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": workload_config(args.workload, wl),
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                             "sample": sample_text(wl, idx, sub) + f", in {k} slices, timed "
                                       f"in {total:.1f} s"},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- our path
def roofline_of(sw, st, workload, sms, f_max, peaks, peak_src, clocks):
    """Roofline of the kernel with the larger share of the step's device time, from the
    library's per-launch CUDA events of the last timed step."""
    inter_cells = st["inter_cells"]
    intra_cells = st["cells"] - inter_cells
    if st["intra_ms"] > st["inter_ms"] and st.get("intra_packed"):
        # packed int16x2 wavefront kernel: two queries per register (batches) or two subjects
        # per register (one query); the same 5.5-operation basis as the inter-task kernels
        kernel = "k_wave_mq_i16x2" if st["intra_packed"] == 1 else "k_wave_ss_i16x2"
        k_ms, k_cells = st["intra_ms"], intra_cells
        peak = sms * LANE_OPS_PER_CLK_SM * f_max * 2.0 / OPS_PER_CELL_PAIR / 1e9
        basis = (f"{sms} SMs x {LANE_OPS_PER_CLK_SM} ALU-pipe int16x2 lane-ops/clk x "
                 f"{f_max / 1e6:.0f} MHz x 2 cells / {OPS_PER_CELL_PAIR} DPX ops per "
                 "cell pair (ALU-pipe bound; HBM is not the bound)")
        rows = None
    elif st["intra_ms"] > st["inter_ms"]:
        kernel, k_ms, k_cells = "k_intra_block_i32", st["intra_ms"], intra_cells
        peak = sms * LANE_OPS_PER_CLK_SM * f_max / ALU_OPS_PER_CELL_I32 / 1e9
        basis = (f"{sms} SMs x {LANE_OPS_PER_CLK_SM} ALU-pipe int32 lane-ops/clk x "
                 f"{f_max / 1e6:.0f} MHz x 1 cell / {ALU_OPS_PER_CELL_I32} DPX ops per cell "
                 "(ALU-pipe bound; HBM is not the bound)")
        rows = None
    else:
        kernel = "k_inter_mq_i16x2" if st.get("multi_query") else "k_inter_i16x2"
        k_ms, k_cells = st["inter_ms"], inter_cells
        peak = sms * LANE_OPS_PER_CLK_SM * f_max * 2.0 / OPS_PER_CELL_PAIR / 1e9
        basis = (f"{sms} SMs x {LANE_OPS_PER_CLK_SM} ALU-pipe int16x2 lane-ops/clk x "
                 f"{f_max / 1e6:.0f} MHz x 2 cells / {OPS_PER_CELL_PAIR} DPX ops per "
                 "cell pair (ALU-pipe bound; HBM is not the bound)")
        rows = INTER_VARIANT_ROWS[st["variant"]]
    achieved = k_cells / (k_ms * 1e-3) / 1e9 if k_ms > 0 else 0.0
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GCUPS",
         "frac": achieved / peak, "traffic": ncu_traffic(workload, kernel, rows),
         "kernel": kernel, "kernel_ms": k_ms, "kernel_cells": int(k_cells),
         "search_device_ms": st["total_ms"],
         "peak_basis": basis, "hbm_peak_gbs": peaks.get("hbm_gbs"), "peaks_source": peak_src}
    if clocks.get("sm_mhz"):
        r["frac_at_observed_clock"] = achieved / (peak * clocks["sm_mhz"] * 1e6 / f_max)
    return r


def dtype_of(st):
    """Arithmetic of the search: int16x2 lanes (exact int32 rescore of saturated lanes) on the
    inter-task kernels and the packed wavefront kernels, int32 on the other intra-task work."""
    inter_cells, cells = st["inter_cells"], st["cells"]
    packed_intra = bool(st.get("intra_packed"))
    if inter_cells == cells or (inter_cells == 0 and packed_intra) or packed_intra:
        return "int16x2 (int32 rescore)"
    if inter_cells == 0:
        return "int32"
    return (f"int16x2 (int32 rescore) for {inter_cells / max(1, cells):.1%} of cells, "
            "int32 for the rest")


def e2e_measure(sw, db, wl, steps, barrier=lambda: None, reduce_max=lambda x: x):
    """The same search through the C ABI with host buffers (pinned): the host->device copy of
    the queries and the device->host copy of every score inside the timed region."""
    import torch
    nq, N = len(wl.queries), db.num_seqs
    h_q = [torch.from_numpy(q).pin_memory() for q in wl.queries]
    h_s = torch.empty(nq * N, dtype=torch.int32).pin_memory()
    arr = (ctypes.POINTER(ctypes.c_uint8) * nq)(
        *[ctypes.cast(t.data_ptr(), ctypes.POINTER(ctypes.c_uint8)) for t in h_q])
    lens = np.array([len(q) for q in wl.queries], np.int32)
    mat = np.ascontiguousarray(wl.matrix, np.int8)
    # the call's arguments are marshalled once, outside the timed loop: each step is the C-ABI
    # call (queries copied in, every score copied out) and a host read of its result
    fn, handle, gap_open, gap_extend = sw.lib.sw_search_batch, db.handle, wl.gap_open, wl.gap_extend
    p_lens = lens.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p_mat = mat.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    p_s = ctypes.cast(h_s.data_ptr(), ctypes.POINTER(ctypes.c_int32))
    h_view = h_s.numpy()

    def e2e_step():
        if fn(handle, arr, p_lens, nq, p_mat, gap_open, gap_extend, p_s) != 0:
            raise RuntimeError(sw.sw_last_error())
        return int(h_view[0])   # read of the step's result on the host

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    dt = reduce_max((time.perf_counter() - t0) / steps)
    return dt, {"h2d_bytes_per_step": int(sum(len(q) for q in wl.queries) + mat.size),
                "d2h_bytes_per_step": int(nq * N * 4)}, h_s.numpy().reshape(nq, N)


def check_rows_golden(got, doc):
    """Every score of every row against the stored oracle row hashes."""
    bad_rows, bad_blocks = [], 0
    blk = doc["block"]
    for q, rec in enumerate(doc["rows"]):
        row = np.ascontiguousarray(got[q], dtype="<i4")
        if sha(row) != rec["sha256"]:
            bad_rows.append(q)
            bad_blocks += sum(sha(row[b:b + blk])[:16] != h
                              for b, h in zip(range(0, row.size, blk), rec["blocks"]))
    n = sum(int(got[q].size) for q in range(len(doc["rows"])))
    return {"ok": not bad_rows, "scores_checked": n,
            "how": "every score: SHA-256 of each int32 score row against the stored oracle row "
                   "hashes (tests/golden/fullsize_batched.json)",
            "bad_rows": bad_rows, "bad_blocks": int(bad_blocks)}


def check_pairs_golden(got, doc):
    pairs = doc["pairs"]
    bad = [(q, d, int(got[q, d]), e) for q, d, e in pairs if int(got[q, d]) != e]
    return {"ok": not bad, "scores_checked": len(pairs),
            "how": "stored oracle scores of a seeded sample of pairs (longest subjects against "
                   "every query, then random pairs)", "mismatches": bad[:5]}


def check_oracle_sample(wl, got, count, seed):
    """Oracle scores of a seeded sample of pairs (the top hit of each query included),
    computed now."""
    import oracle
    rng = np.random.default_rng(seed)
    nq, n = got.shape
    pairs = {(int(rng.integers(nq)), int(rng.integers(n))) for _ in range(count)}
    pairs |= {(q, int(np.argmax(got[q]))) for q in range(nq)}
    pairs = sorted(pairs)
    qsel = np.array([p[0] for p in pairs], np.int64)
    dsel = np.array([p[1] for p in pairs], np.int64)
    exp = oracle.sw_pairs(wl.queries, wl.db.residues, wl.db.offsets, qsel, dsel, wl.matrix,
                          wl.gap_open, wl.gap_extend)
    bad = [(p, int(got[p]), int(e)) for p, e in zip(pairs, exp) if got[p] != e]
    return {"ok": not bad, "scores_checked": len(pairs),
            "how": "oracle recomputation of a seeded sample of pairs (top hit of every query "
                   "included)", "mismatches": bad[:5]}


def check_oracle_all(wl, got):
    import oracle
    bad, cores, oracle_s, threads = 0, 0, 0.0, host_cores()
    for q in range(len(wl.queries)):
        t0 = time.perf_counter()
        exp, cores = oracle.sw_search(wl.queries[q], wl.db.residues, wl.db.offsets, wl.matrix,
                                      wl.gap_open, wl.gap_extend, threads=threads)
        oracle_s += time.perf_counter() - t0
        bad += int(np.count_nonzero(got[q].astype(np.int64) != exp))
    return {"ok": bad == 0, "scores_checked": int(got.size),
            "how": "every score recomputed by the oracle", "mismatches": bad,
            "oracle_s": round(oracle_s, 3), "oracle_cores": int(cores)}


# fixed seeded samples of database sequences for the oracle timing of the larger configurations
# (15-25 s of CPU work each on 16 cores): 0.1 % of the paper-shaped database, 16 of the
# long-subject database's 50,000 subjects (each 5,000-35,000 residues)
CONFIG_CPU_SAMPLE = {"paper_shaped": lambda n: max(16, int(round(n * 0.001))),
                     "long_subject": lambda n: min(n, 16)}


def config_cpu_baseline(name, wl, par):
    """The oracle timed on a configuration: the whole plain configuration (its parity check runs
    the oracle over every score), a fixed seeded sample of the larger databases."""
    cells_q = sum(len(q) for q in wl.queries)
    if name == "plain" and "oracle_s" in par:
        return {"value": cells_q * wl.db.num_residues / par["oracle_s"] / 1e9, "unit": "GCUPS",
                "cores": par["oracle_cores"], "kind": "oracle",
                "sample": f"the whole configuration ({wl.db.num_seqs} sequences, "
                          f"{cells_q * wl.db.num_residues:.3e} cells), timed in {par['oracle_s']:.2f} s"}
    if name not in CONFIG_CPU_SAMPLE:
        return None
    n = wl.db.num_seqs
    idx = w.sample_indices(n, CONFIG_CPU_SAMPLE[name](n), seed=CPU_SAMPLE_SEED)
    sub = wl.db.subset(idx)
    dt, cores = time_oracle(wl, sub)
    cells = cells_q * sub.num_residues
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": f"all {len(wl.queries)} queries vs a fixed seeded sample of the database "
                      f"(seed {CPU_SAMPLE_SEED}: {len(idx)} of {n} sequences, {cells:.3e} cells), "
                      f"timed in {dt:.1f} s"}


def parity(name, wl, got):
    doc = load_golden(name, wl)
    if doc is not None and "rows" in doc:
        return check_rows_golden(got, doc)
    if name == "plain":
        return check_oracle_all(wl, got)
    out = check_pairs_golden(got, doc) if doc is not None else {"ok": True, "scores_checked": 0}
    extra = check_oracle_sample(wl, got, 64, seed=5)
    out["ok"] = out["ok"] and extra["ok"]
    out["scores_checked"] += extra["scores_checked"]
    out["mismatches"] = (out.get("mismatches", []) + extra["mismatches"])[:5]
    out["how"] = (out.get("how", "") + "; " if doc is not None else "") + extra["how"]
    return out


class Search:
    """A loaded workload: database handle, device buffers, the timed step."""

    def __init__(self, sw, name, wl, args, tune=True):
        import torch
        self.sw, self.name, self.wl = sw, name, wl
        nq = len(wl.queries)
        cat = np.concatenate(wl.queries)
        self.qoff = np.zeros(nq + 1, np.int64)
        np.cumsum([len(q) for q in wl.queries], out=self.qoff[1:])
        # inter-task cutoff: the library default (3,072) except on the paper-shaped database,
        # whose heavy tail runs faster with subjects up to 6,144 residues on the int16x2 kernel
        self.cutoff = args.long_cutoff or (6144 if name == "paper_shaped" else 0)
        self.db = sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE,
                                long_cutoff=self.cutoff,
                                placement=sw.PLACE_HOST if args.placement == "host"
                                else sw.PLACE_DEVICE)
        self.N = self.db.num_seqs
        self.d_q = torch.from_numpy(cat).cuda()
        self.d_s = torch.empty(nq * self.N, dtype=torch.int32, device="cuda")
        self.stream = torch.cuda.current_stream()
        self.cells = int(cat.size) * wl.db.num_residues
        self.tune = None
        if args.variant >= 0:
            sw.sw_db_set_variant(self.db, args.variant)
            self.tune = {"variant": args.variant, "forced": True}
        elif tune and not args.no_tune and nq >= 1 and self.N >= 100000:
            # probe: the two median-length queries (the batch kernel pairs queries) against the
            # whole database, every kernel variant
            srt = sorted(wl.queries, key=len)
            probe = srt[max(0, len(srt) // 2 - 1): len(srt) // 2 + 1]
            self.tune = sw.sw_db_tune(self.db, probe, wl.matrix, wl.gap_open, wl.gap_extend)

    def step(self):
        self.sw.sw_search_batch_device(self.db, self.d_q, self.qoff, self.wl.matrix,
                                       self.wl.gap_open, self.wl.gap_extend, self.d_s,
                                       stream=self.stream)

    def timed(self, warmup, steps, sampler, barrier=lambda: None):
        import torch
        for _ in range(warmup):
            self.step()
        torch.cuda.synchronize()
        with Timed(sampler) as tr:
            barrier()
            torch.cuda.synchronize()
            launches0 = self.sw.sw_launch_count()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(self.stream)
            for _ in range(steps):
                self.step()              # asynchronous: steps queue back to back
            ev1.record(self.stream)
            torch.cuda.synchronize()
            st = self.sw.sw_get_stats(self.db)   # per-kernel CUDA events of the last step
            barrier()
            launches = self.sw.sw_launch_count() - launches0
        return ev0.elapsed_time(ev1) / steps, st, launches, tr.clocks

    def scores(self):
        return self.d_s.cpu().numpy().reshape(len(self.wl.queries), self.N)

    def close(self):
        self.db.close()


def one_query_per_launch(sw, s, args):
    """The same queries, one query per launch (the plain search): same kernels, no batching."""
    import torch
    wl, db = s.wl, s.db
    plain_variant = None
    if args.variant < 0 and not args.no_tune:
        # the single-query kernel gets its own tuned variant (the batch run's variant was tuned
        # for the two-queries-per-register kernel); restored after the comparison
        med = sorted(wl.queries, key=len)[len(wl.queries) // 2]
        plain_variant = sw.sw_db_tune(db, [med], wl.matrix, wl.gap_open, wl.gap_extend)
    offs1 = [np.array([0, len(q)], np.int64) for q in wl.queries]
    d_qs = [torch.from_numpy(q).cuda() for q in wl.queries]
    d_s1 = torch.empty(s.N, dtype=torch.int32, device="cuda")

    def plain_step():
        for dq, o in zip(d_qs, offs1):
            sw.sw_search_batch_device(db, dq, o, wl.matrix, wl.gap_open, wl.gap_extend, d_s1,
                                      stream=s.stream)

    plain_step()
    torch.cuda.synchronize()
    # one event per query boundary: the pass's total and each query's own time
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(wl.queries) + 1)]
    evs[0].record(s.stream)
    for k, (dq, o) in enumerate(zip(d_qs, offs1)):
        sw.sw_search_batch_device(db, dq, o, wl.matrix, wl.gap_open, wl.gap_extend, d_s1,
                                  stream=s.stream)
        evs[k + 1].record(s.stream)
    torch.cuda.synchronize()
    p_ms = evs[0].elapsed_time(evs[-1])
    per_len = []
    for k, q in enumerate(wl.queries):
        q_ms = evs[k].elapsed_time(evs[k + 1])
        per_len.append({"m": len(q), "ms": round(q_ms, 3),
                        "gcups": round(len(q) * wl.db.num_residues / (q_ms * 1e-3) / 1e9, 1)})
    out = {"gcups": s.cells / (p_ms * 1e-3) / 1e9, "ms_per_pass": p_ms,
           "what": "the same queries, one per launch (single-query kernel)",
           "kernel_variant": plain_variant, "per_query_length": per_len}
    if args.score_profile:
        # the same pass with the score profile (Section 4.3) in place of the query profile
        os.environ["SWGB_SCORE_PROFILE"] = "1"
        plain_step()
        torch.cuda.synchronize()
        sp_used = sw.sw_get_stats(db)["score_profile"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        plain_step()
        e1.record(s.stream)
        torch.cuda.synchronize()
        del os.environ["SWGB_SCORE_PROFILE"]
        sp_ms = e0.elapsed_time(e1)
        out["score_profile"] = {"gcups": s.cells / (sp_ms * 1e-3) / 1e9, "ms_per_pass": sp_ms,
                                "kernel_used": bool(sp_used)}
    if plain_variant is not None and s.tune is not None:
        sw.sw_db_set_variant(db, s.tune["variant"])
    return out


def measure_extra(sw, name, args, sampler, sms, f_max, peaks, peak_src):
    """One of the other workloads: GCUPS, dominant kernel's roofline, e2e, oracle check."""
    import torch
    t_gen = time.perf_counter()
    wl = make_workload(name, args.seed, args.scale)
    s = Search(sw, name, wl, args)
    setup_s = time.perf_counter() - t_gen
    try:
        warm, steps, e2e_steps = EXTRA_STEPS[name]
        ms, st, launches, clocks = s.timed(warm, steps, sampler)
        got = s.scores()
        out = {"config": workload_config(name, wl), "value": s.cells / (ms * 1e-3) / 1e9,
               "unit": "GCUPS", "ms_per_step": ms, "steps": steps, "warmup": warm,
               "dtype": dtype_of(st), "gpu_launches": int(launches),
               "kernel_variant": s.tune, "long_cutoff": s.cutoff or 3072,
               "roofline": roofline_of(sw, st, name, sms, f_max, peaks, peak_src, clocks),
               "clocks": clocks, "flagged_lanes_per_step": st["flagged"],
               "setup_s": round(setup_s, 1)}
        if not args.no_e2e:
            dt, io, h_got = e2e_measure(sw, s.db, wl, e2e_steps)
            out["e2e"] = {"value": s.cells / dt / 1e9, "unit": "GCUPS", **io}
            if not np.array_equal(h_got, got):
                out["e2e"]["mismatch_vs_device_path"] = True
        out["parity"] = parity(name, wl, got)
        if not args.no_cpu_baseline:
            cb = config_cpu_baseline(name, wl, out["parity"])
            if cb is not None:
                out["cpu_baseline"] = cb
        torch.cuda.synchronize()
        return out
    finally:
        s.close()
        del s, wl


def measure_serving(sw, s, args, sampler):
    """Continuous-batching server on the resident headline database: capacity (a burst of 48
    requests), then Poisson arrivals at fractions of it; every request's scores at a seeded
    sample of sequences are checked against the oracle."""
    import oracle
    db, wl = s.db, s.wl
    srv = sw.Server(db, wl.matrix, wl.gap_open, wl.gap_extend, max_inflight=32,
                    slices=args.slices)
    checked, bad = 0, []
    rng = np.random.default_rng(77)
    try:
        burst = w.serving_queries(48, seed=args.seed + 100)
        for t in [srv.submit(q) for q in burst[:8]]:      # warm-up
            srv.wait(t, 600000)
        srv.stats(reset=True)
        with Timed(sampler) as tr:
            t0 = time.perf_counter()
            for t in [srv.submit(q) for q in burst]:
                srv.wait(t, 600000)
            cap_s = time.perf_counter() - t0
        capacity = len(burst) / cap_s
        cap_stats = srv.stats(reset=True)
        results = []
        for i, frac in enumerate(float(x) for x in args.rates.split(",") if x):
            rate = frac * capacity
            qs = w.serving_queries(args.requests, seed=args.seed + 200 + i)
            arrivals = w.poisson_arrivals(args.requests, rate, seed=args.seed + 300 + i)
            tickets = []
            with Timed(sampler) as tr:
                start = time.perf_counter()
                for a, q in zip(arrivals, qs):
                    delay = start + a - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                    tickets.append(srv.submit(q))
                outs = [srv.wait(t, 600000) for t in tickets]
            st = srv.stats(reset=True)
            # oracle check: 16 seeded sequences of every request
            sel = rng.choice(s.N, size=16, replace=False)
            qsel = np.repeat(np.arange(len(qs)), sel.size)
            dsel = np.tile(sel, len(qs))
            exp = oracle.sw_pairs(qs, wl.db.residues, wl.db.offsets, qsel, dsel, wl.matrix,
                                  wl.gap_open, wl.gap_extend)
            gotv = np.array([outs[q][d] for q, d in zip(qsel, dsel)], np.int64)
            checked += int(exp.size)
            bad += [(int(q), int(d)) for q, d in zip(qsel[gotv != exp], dsel[gotv != exp])]
            results.append({"rate_frac": frac, "rate_rps": rate, "requests": args.requests,
                            "p50_ms": st["latency_p50_ms"], "p99_ms": st["latency_p99_ms"],
                            "mean_ms": st["latency_mean_ms"], "max_ms": st["latency_max_ms"],
                            "gcups": st["gcups"], "max_in_flight": st["max_in_flight"],
                            "joined_while_running": st["joined_while_running"],
                            "ticks": st["ticks"], "clocks": tr.clocks})
    finally:
        srv.close()
    return {"config": {"workload": WORKLOAD_TEXT["serving"], "db_seqs": s.N,
                       "db_residues": wl.db.num_residues, "max_inflight": 32,
                       "slices": args.slices if args.slices > 0 else "auto",
                       "requests_per_rate": args.requests},
            "capacity_rps": capacity, "capacity_gcups": cap_stats["gcups"],
            "capacity_p50_ms": cap_stats["latency_p50_ms"],
            "capacity_p99_ms": cap_stats["latency_p99_ms"],
            "sustained_gcups": max((r["gcups"] for r in results), default=0.0),
            "rates": results, "unit": "GCUPS / ms",
            "parity": {"ok": not bad, "scores_checked": checked,
                       "how": "oracle recomputation of 16 seeded sequences of every request",
                       "mismatches": bad[:5]}}


def run_ours(args, world, rank, local):
    import torch
    import paper_1702_07195_gb300 as sw

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def reduce_max(x):
        if dist is None:
            return x
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    name = args.workload
    wl = make_workload(name, args.seed + rank, args.scale, args.query_lengths)
    s = Search(sw, name, wl, args)
    sampler = ClockSampler(local)
    ms, st, launches, clocks_head = s.timed(args.warmup, args.steps, sampler, barrier)
    t_max = reduce_max(ms)
    # units all ranks processed (each rank's database has its own seed, so sizes differ slightly)
    cells_all = s.cells
    if dist is not None:
        c = torch.tensor([s.cells], dtype=torch.int64, device="cuda")
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        cells_all = int(c.item())
    value = cells_all / (t_max * 1e-3) / 1e9
    got = s.scores() if rank == 0 and world == 1 else None

    e2e = None
    if not args.no_e2e:
        dt, io, _ = e2e_measure(sw, s.db, wl, args.steps, barrier, reduce_max)
        e2e = {"value": cells_all / dt / 1e9, "unit": "GCUPS", **io}

    plain = None
    if not args.no_plain and len(wl.queries) > 1:
        plain = one_query_per_launch(sw, s, args)

    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    f_max = float(clocks_head.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)) * 1e6

    extras = {}
    do_extra = world == 1 and not args.headline_only and name == "batched" and args.scale == 1.0 \
        and not args.query_lengths
    wanted = [x for x in args.extra.split(",") if x] if do_extra else []
    if "serving" in wanted:
        try:
            extras["serving"] = measure_serving(sw, s, args, sampler)
        except Exception as exc:   # recorded in the line; the headline stands
            extras["serving"] = {"error": repr(exc)}
    s.close()
    for xname in ("plain", "long_subject", "paper_shaped"):
        if xname in wanted:
            try:
                extras[xname] = measure_extra(sw, xname, args, sampler, sms, f_max, peaks,
                                              peak_src)
            except Exception as exc:
                extras[xname] = {"error": repr(exc)}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    line = {"metric": "GCUPS", "value": value, "unit": "GCUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(st), "data": "synthetic",
            "config": workload_config(name, wl),
            "run": {"kernel_variant": s.tune, "placement": args.placement,
                    "long_cutoff": s.cutoff or 3072, "cells_per_step": s.cells,
                    "cells_per_step_all_ranks": cells_all,
                    "per_gpu": "each rank searches its own database of this size"},
            "roofline": roofline_of(sw, st, name, sms, f_max, peaks, peak_src, clocks_head),
            "clocks": sampler.summary(), "clocks_headline": clocks_head,
            "gpu_launches": int(launches),
            "plain_one_query_per_launch": plain,
            "flagged_lanes_per_step": st["flagged"]}
    if e2e:
        line["e2e"] = e2e
    if got is not None:
        line["parity"] = parity(name, wl, got)
    if extras:
        line["configs"] = extras
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_serving(args, world, rank, local):
    """Serving alone (--workload serving): the same measurement as the default line's
    "serving" entry, as a line of its own."""
    import torch
    import paper_1702_07195_gb300 as sw

    torch.cuda.set_device(local)
    wl = make_workload("batched", args.seed + rank, args.scale)
    s = Search(sw, "batched", wl, args)
    sampler = ClockSampler(local)
    res = measure_serving(sw, s, args, sampler)
    s.close()
    line = {"metric": "GCUPS (served)", "value": res["sustained_gcups"], "unit": "GCUPS",
            "n_gpus": world, "steps": len(res["rates"]), "warmup": 1, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int16x2 (int32 rescore)", "data": "synthetic", "config": res["config"],
            "serving": res, "clocks": sampler.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "serving":
        run_serving(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
