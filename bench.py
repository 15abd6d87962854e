"""Benchmark: GCUPS of the Smith-Waterman database search on GB300.

One step = one pass of the whole search (query profiles, inter-task int16x2 kernel,
intra-task kernel for long subjects, int32 rescore of saturated lanes) for a batch of
queries against the device-resident database.  Default workload: the 20 paper-shaped query
lengths (144..5478, sum 30,747) against a seeded synthetic database of 1M protein
sequences (log-normal lengths, mean 250, clipped to 20..2000; ~249M residues), BLOSUM62,
a gap of length k costing 10 + 2(k - 1).  GCUPS = sum(|Q|) * |D| / (t * 1e9) (paper
Eq. gcups).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank searches its own database of the
same size (weak scaling; no collective on the data path).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
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

# ALU-pipe roofline of the inter-task kernel: the DPX max-plus
# operations issue on the ALU pipe at 64 lane-operations per clock per SM (ncu: the pipe is
# 92% busy at 0.52 IPC per sub-partition; wall-clock probe: 18.9e12 lane-ops/s at 2,070 MHz
# on 152 SMs), two cells per int16x2 lane-operation, and at least 5.5 ALU operations per cell
# pair for Eqs. sw2-sw4 (5 DPX updates + half a three-way max for the running best).
LANE_OPS_PER_CLK_SM = 64
OPS_PER_CELL_PAIR = 5.5
# int32 update: 4 viaddmax + half a vimax3 per cell on the ALU pipe; the subtraction of Goe is a
# plain integer add, which issues on the FMA pipe
ALU_OPS_PER_CELL_I32 = 4.5
INTER_KERNEL = "k_inter_i16x2"
INTER_SRC = os.path.join(ROOT, "paper_1702_07195_gb300", "csrc", "k_inter.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "plain", "paper_shaped", "long_subject", "serving",
                             "simd_rates"])
    ap.add_argument("--requests", type=int, default=200, help="serving: requests per rate")
    ap.add_argument("--slices", type=int, default=0,
                    help="serving: database slices per scan cycle (0: automatic)")
    ap.add_argument("--rates", default="0.25,0.5,0.9,1.1",
                    help="serving: arrival rates as fractions of the measured capacity")
    ap.add_argument("--scale", type=float, default=1.0, help="database scale (tests only)")
    ap.add_argument("--query-lengths", default="",
                    help="comma-separated query lengths replacing the workload's (profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="skip the kernel-variant autotuner")
    ap.add_argument("--variant", type=int, default=-1,
                    help="force an inter-task kernel variant instead of autotuning (profiling)")
    ap.add_argument("--long-cutoff", type=int, default=0,
                    help="subjects longer than this go to the intra-task kernel (0: library default)")
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


def make_workload(name, seed, scale, query_lengths=""):
    if name == "serving":
        name = "batched"
    if query_lengths:
        ql = [int(x) for x in query_lengths.split(",") if x]
        return getattr(w, name)(seed=seed, scale=scale, query_lengths=ql)
    return getattr(w, name)(seed=seed, scale=scale)


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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


# ---------------------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


KERNEL_SRC = {"k_inter_i16x2": INTER_SRC,
              "k_inter_mq_i16x2": os.path.join(ROOT, "paper_1702_07195_gb300", "csrc",
                                               "k_inter_mq.cu"),
              "k_intra_block_i32": os.path.join(ROOT, "paper_1702_07195_gb300", "csrc",
                                                "k_intra_block.cu")}


# rows per strip of the inter-task kernel variants (both kernels), as in csrc/k_inter*.cu
INTER_VARIANT_ROWS = (32, 64, 32, 64)


def ncu_traffic(workload, kernel=INTER_KERNEL, rows_per_strip=None):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None
    if the summary is absent, was taken on a different kernel source, or (for the inter-task
    kernels, whose boundary traffic scales with the strip count) on another strip height."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
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


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------- oracle baseline
def cpu_baseline(wl, seconds, seed):
    """The oracle (as it stands) on the host cores, on a seeded sample of the database sized
    for about `seconds` of CPU work.  Returns the cpu_baseline dict."""
    import oracle
    oracle.build()
    total_m = sum(len(q) for q in wl.queries)
    n = wl.db.num_seqs
    # calibrate on a small sample
    probe = w.sample_indices(n, min(n, 200), seed=seed + 1)
    sub = wl.db.subset(probe)
    t0 = time.perf_counter()
    _, cores = oracle.sw_search(wl.queries[0], sub.residues, sub.offsets, wl.matrix,
                                wl.gap_open, wl.gap_extend)
    dt = max(time.perf_counter() - t0, 1e-4)
    rate = len(wl.queries[0]) * sub.num_residues / dt
    want_res = max(1, int(rate * seconds / total_m))
    mean_len = max(1.0, wl.db.num_residues / max(1, n))
    count = int(min(n, max(16, want_res / mean_len)))
    idx = w.sample_indices(n, count, seed=seed + 2)
    sub = wl.db.subset(idx)
    t0 = time.perf_counter()
    for q in wl.queries:
        oracle.sw_search(q, sub.residues, sub.offsets, wl.matrix, wl.gap_open, wl.gap_extend)
    dt = time.perf_counter() - t0
    cells = total_m * sub.num_residues
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": int(cores), "kind": "oracle",
            "sample": f"all {len(wl.queries)} queries vs a seeded sample of {count} of the "
                      f"{n} database sequences ({sub.num_residues} residues, {cells:.3e} cells,"
                      f" {dt:.1f} s)",
            "seconds": dt}


def run_reference(args, world, rank):
    if rank != 0:
        return
    wl = make_workload(args.workload, args.seed, args.scale, args.query_lengths)
    vals = []
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    cb = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(wl, per_step, args.seed + 17 * i)
        if i >= args.warmup:
            vals.append(cb["value"])
    value = statistics.mean(vals) if vals else cb["value"]
    cb["value"] = value
    line = {"impl": "reference", "metric": "GCUPS", "value": value, "unit": "GCUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * cb["seconds"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload],
                       "queries": len(wl.queries), "db_seqs": wl.db.num_seqs,
                       "db_residues": wl.db.num_residues},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- our path
def run_ours(args, world, rank, local):
    import torch
    import paper_1702_07195_gb300 as sw

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = make_workload(args.workload, args.seed + rank, args.scale, args.query_lengths)
    nq = len(wl.queries)
    cat = np.concatenate(wl.queries)
    qoff = np.zeros(nq + 1, np.int64)
    np.cumsum([len(q) for q in wl.queries], out=qoff[1:])
    # inter-task cutoff: the library default (3,072) except on the paper-shaped database, whose
    # heavy tail runs faster with subjects up to 6,144 residues on the int16x2 kernel (6,391 ->
    # 6,483 GCUPS; 12,288: 6,454)
    cutoff = args.long_cutoff or (6144 if args.workload == "paper_shaped" else 0)
    db = sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE, long_cutoff=cutoff,
                       placement=sw.PLACE_HOST if args.placement == "host" else sw.PLACE_DEVICE)
    N = db.num_seqs
    d_q = torch.from_numpy(cat).cuda()
    d_s = torch.empty(nq * N, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    cells = int(cat.size) * wl.db.num_residues

    tune = None
    if args.variant >= 0:
        sw.sw_db_set_variant(db, args.variant)
        tune = {"variant": args.variant, "forced": True}
    elif not args.no_tune:
        # probe: the two median-length queries (the batch kernel pairs queries) against the
        # whole database, every kernel variant
        srt = sorted(wl.queries, key=len)
        probe = srt[max(0, len(srt) // 2 - 1): len(srt) // 2 + 1]
        tune = sw.sw_db_tune(db, probe, wl.matrix, wl.gap_open, wl.gap_extend)

    def step():
        sw.sw_search_batch_device(db, d_q, qoff, wl.matrix, wl.gap_open, wl.gap_extend, d_s,
                                  stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    launches0 = sw.sw_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()                            # asynchronous: steps queue back to back
    ev1.record(stream)
    torch.cuda.synchronize()
    # per-kernel CUDA events (on the launch stream) of the last timed step
    st_timed = sw.sw_get_stats(db)
    inter_ms, intra_ms = [st_timed["inter_ms"]], [st_timed["intra_ms"]]
    flagged = st_timed["flagged"] * args.steps
    barrier()
    launches = sw.sw_launch_count() - launches0
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    t_max = ms
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    # units all ranks processed (each rank's database has its own seed, so sizes differ slightly)
    cells_all = cells
    if dist is not None:
        c = torch.tensor([cells], dtype=torch.int64, device="cuda")
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        cells_all = int(c.item())
    value = cells_all / (t_max * 1e-3) / 1e9

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_q = [torch.from_numpy(q).pin_memory() for q in wl.queries]
        h_s = torch.empty(nq * N, dtype=torch.int32).pin_memory()
        import ctypes
        arr = (ctypes.POINTER(ctypes.c_uint8) * nq)(
            *[ctypes.cast(t.data_ptr(), ctypes.POINTER(ctypes.c_uint8)) for t in h_q])
        lens = np.array([len(q) for q in wl.queries], np.int32)
        mat = np.ascontiguousarray(wl.matrix, np.int8)

        def e2e_step():
            s = sw.lib.sw_search_batch(db.handle, arr, lens.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       nq, mat.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                       wl.gap_open, wl.gap_extend,
                                       ctypes.cast(h_s.data_ptr(), ctypes.POINTER(ctypes.c_int32)))
            if s != 0:
                raise RuntimeError(sw.sw_last_error())
            return int(h_s[0])   # read of the step's result on the host

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        dt = (time.perf_counter() - t0) / args.steps
        if dist is not None:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": cells_all / dt / 1e9, "unit": "GCUPS",
               "h2d_bytes_per_step": int(cat.size + mat.size),
               "d2h_bytes_per_step": int(nq * N * 4)}

    # the same queries, one query per launch (the "plain" search): same kernels, no batching
    plain = None
    if not args.no_plain and nq > 1:
        # the single-query kernel gets its own tuned variant (the batch run's variant was tuned
        # for the two-queries-per-register kernel); restored after the comparison
        plain_variant = None
        if args.variant < 0 and not args.no_tune:
            med = sorted(wl.queries, key=len)[len(wl.queries) // 2]
            plain_variant = sw.sw_db_tune(db, [med], wl.matrix, wl.gap_open, wl.gap_extend)
        offs1 = [np.array([0, len(q)], np.int64) for q in wl.queries]
        d_qs = [torch.from_numpy(q).cuda() for q in wl.queries]
        d_s1 = torch.empty(N, dtype=torch.int32, device="cuda")

        def plain_step():
            for dq, o in zip(d_qs, offs1):
                sw.sw_search_batch_device(db, dq, o, wl.matrix, wl.gap_open, wl.gap_extend, d_s1,
                                          stream=stream)

        plain_step()
        torch.cuda.synchronize()
        # one event per query boundary: the pass's total and each query's own time
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(nq + 1)]
        evs[0].record(stream)
        for k, (dq, o) in enumerate(zip(d_qs, offs1)):
            sw.sw_search_batch_device(db, dq, o, wl.matrix, wl.gap_open, wl.gap_extend, d_s1,
                                      stream=stream)
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
        p_ms = evs[0].elapsed_time(evs[-1])
        per_len = []
        for k, q in enumerate(wl.queries):
            q_ms = evs[k].elapsed_time(evs[k + 1])
            per_len.append({"m": len(q), "ms": round(q_ms, 3),
                            "gcups": round(len(q) * wl.db.num_residues / (q_ms * 1e-3) / 1e9, 1)})
        plain = {"gcups": cells / (p_ms * 1e-3) / 1e9, "ms_per_pass": p_ms,
                 "what": "the same queries, one per launch (single-query kernel)",
                 "kernel_variant": plain_variant, "per_query_length": per_len}
        if args.score_profile:
            # the same pass with the score profile (Section 4.3) in place of the query profile
            os.environ["SWGB_SCORE_PROFILE"] = "1"
            plain_step()
            torch.cuda.synchronize()
            sp_used = sw.sw_get_stats(db)["score_profile"]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plain_step()
            e1.record(stream)
            torch.cuda.synchronize()
            del os.environ["SWGB_SCORE_PROFILE"]
            sp_ms = e0.elapsed_time(e1)
            plain["score_profile"] = {"gcups": cells / (sp_ms * 1e-3) / 1e9, "ms_per_pass": sp_ms,
                                      "kernel_used": bool(sp_used)}
        if plain_variant is not None and tune is not None:
            sw.sw_db_set_variant(db, tune["variant"])

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    f_max = float(clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_gcups = sms * LANE_OPS_PER_CLK_SM * f_max * 2.0 / OPS_PER_CELL_PAIR / 1e9
    st_last = st_timed if st_timed is not None else sw.sw_get_stats(db)
    inter_cells = st_last["inter_cells"]
    intra_cells = st_last["cells"] - inter_cells
    inter_k_ms = statistics.mean(inter_ms) if inter_ms else 0.0
    intra_k_ms = statistics.mean(intra_ms) if intra_ms else 0.0
    # the dominant kernel: the one with the larger share of the step's device time
    if intra_k_ms > inter_k_ms:
        kernel_name, k_ms, k_cells = "k_intra_block_i32", intra_k_ms, intra_cells
        peak_gcups = sms * LANE_OPS_PER_CLK_SM * f_max / ALU_OPS_PER_CELL_I32 / 1e9
        basis = (f"{sms} SMs x {LANE_OPS_PER_CLK_SM} ALU-pipe int32 lane-ops/clk x "
                 f"{f_max / 1e6:.0f} MHz x 1 cell / {ALU_OPS_PER_CELL_I32} DPX ops per cell "
                 "(ALU-pipe bound; HBM is not the bound)")
    else:
        kernel_name = "k_inter_mq_i16x2" if st_last.get("multi_query") else INTER_KERNEL
        k_ms, k_cells = inter_k_ms, inter_cells
        basis = (f"{sms} SMs x {LANE_OPS_PER_CLK_SM} ALU-pipe int16x2 lane-ops/clk x "
                 f"{f_max / 1e6:.0f} MHz x 2 cells / {OPS_PER_CELL_PAIR} DPX ops per "
                 "cell pair (ALU-pipe bound; HBM is not the bound)")
    achieved = k_cells / (k_ms * 1e-3) / 1e9 if k_ms > 0 else 0.0
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_gcups, "unit": "GCUPS",
                "frac": achieved / peak_gcups,
                "traffic": ncu_traffic(args.workload, kernel_name,
                                       INTER_VARIANT_ROWS[st_last["variant"]]
                                       if kernel_name.startswith("k_inter") else None),
                "kernel": kernel_name, "kernel_ms": k_ms, "kernel_cells": int(k_cells),
                "peak_basis": basis,
                "hbm_peak_gbs": peaks.get("hbm_gbs"), "peaks_source": peak_src}
    dtype = ("int32" if inter_cells == 0 else
             "int16x2 (int32 rescore)" if intra_cells == 0 else
             f"int16x2 (int32 rescore) for {inter_cells / max(1, st_last['cells']):.1%} of cells, "
             "int32 for the rest")
    if clocks.get("sm_mhz"):
        roofline["frac_at_observed_clock"] = achieved / (peak_gcups * clocks["sm_mhz"] * 1e6 / f_max)
    line = {"metric": "GCUPS", "value": value, "unit": "GCUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "queries": nq,
                       "query_residues": int(cat.size), "db_seqs": N,
                       "db_residues": wl.db.num_residues, "cells_per_step": cells,
                       "cells_per_step_all_ranks": cells_all,
                       "kernel_variant": tune,
                       "per_gpu": "each rank searches its own database of this size",
                       "placement": args.placement, "long_cutoff": cutoff or 3072,
                       "l2": f"inputs larger than L2 (database {wl.db.num_residues / 1e6:.0f} MB "
                             "resident in HBM, read once per query per step)"},
            "roofline": roofline, "clocks": clocks, "gpu_launches": int(launches),
            "plain_one_query_per_launch": plain,
            "flagged_lanes_per_step": flagged / max(1, args.steps)}
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_baseline(wl, args.cpu_seconds, args.seed)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line), flush=True)
    db.close()
    if dist is not None:
        dist.destroy_process_group()


def run_serving(args, world, rank, local):
    """Continuous-batching server under Poisson arrivals at several rates."""
    import torch
    import paper_1702_07195_gb300 as sw

    torch.cuda.set_device(local)
    wl = make_workload("batched", args.seed + rank, args.scale)
    db = sw.sw_db_load(wl.db.residues, wl.db.offsets, w.ALPHABET_SIZE)
    R = wl.db.num_residues
    probe = w.serving_queries(2, seed=args.seed + 50)
    tune = sw.sw_db_tune(db, probe, wl.matrix, wl.gap_open, wl.gap_extend)
    srv = sw.Server(db, wl.matrix, wl.gap_open, wl.gap_extend, max_inflight=32, slices=args.slices)
    # capacity: a burst of requests submitted together
    burst = w.serving_queries(48, seed=args.seed + 100)
    for t in [srv.submit(q) for q in burst[:8]]:      # warm-up
        srv.wait(t, 600000)
    srv.stats(reset=True)
    t0 = time.perf_counter()
    for t in [srv.submit(q) for q in burst]:
        srv.wait(t, 600000)
    cap_s = time.perf_counter() - t0
    capacity = len(burst) / cap_s
    cap_stats = srv.stats(reset=True)
    results = []
    sampler = ClockSampler(local)
    sampler.start()
    for i, frac in enumerate(float(x) for x in args.rates.split(",") if x):
        rate = frac * capacity
        qs = w.serving_queries(args.requests, seed=args.seed + 200 + i)
        arrivals = w.poisson_arrivals(args.requests, rate, seed=args.seed + 300 + i)
        tickets = []
        start = time.perf_counter()
        for a, q in zip(arrivals, qs):
            delay = start + a - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(q))
        for t in tickets:
            srv.wait(t, 600000)
        st = srv.stats(reset=True)
        results.append({"rate_frac": frac, "rate_rps": rate, "requests": args.requests,
                        "p50_ms": st["latency_p50_ms"], "p99_ms": st["latency_p99_ms"],
                        "mean_ms": st["latency_mean_ms"], "gcups": st["gcups"],
                        "max_in_flight": st["max_in_flight"],
                        "joined_while_running": st["joined_while_running"],
                        "ticks": st["ticks"]})
    clocks = sampler.stop()
    srv.close()
    db.close()
    best = max((r for r in results if r["rate_frac"] <= 1.0), key=lambda r: r["gcups"],
               default=results[-1] if results else {"gcups": 0.0})
    line = {"metric": "GCUPS (served)", "value": best["gcups"], "unit": "GCUPS", "n_gpus": world,
            "steps": len(results), "warmup": 1, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int16x2 (int32 rescore)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT["serving"], "db_seqs": wl.db.num_seqs,
                       "db_residues": R, "max_inflight": 32,
                       "slices": args.slices if args.slices > 0 else "auto",
                       "kernel_variant": tune,
                       "capacity_rps": capacity, "capacity_gcups": cap_stats["gcups"]},
            "serving": results, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_simd_rates(args, rank):
    """The int8-tier study (Section 4.2's 8-bit first tier): rates of the packed-integer
    operations a cell update can be built from, measured by the probe that build() compiles,
    and the cell-update rates they bound (int16x2 DPX vs 4 x 8-bit SIMD)."""
    if rank != 0:
        return
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_swgb_build", os.path.join(ROOT, "paper_1702_07195_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    r = subprocess.run([b.PROBE], capture_output=True, text=True, timeout=300)
    probe = json.loads(r.stdout.strip().splitlines()[-1])
    if r.returncode != 0 or "error" in probe:
        raise RuntimeError(f"probe failed: {r.stdout} {r.stderr}")
    cu = probe["cell_updates_per_s"]
    print(json.dumps({"metric": "cell-update rate bound from packed-integer operation rates",
                      "value": cu["int16x2_dpx"] / 1e9, "unit": "GCUPS", "n_gpus": 1,
                      "higher_is_better": True, "dtype": "int16x2 vs int8x4", "data": "synthetic",
                      "config": {"workload": "simd_rates"},
                      "int8x4_simd_gcups_bound": cu["int8x4_simd"] / 1e9,
                      "int16x2_over_int8x4": cu["int16x2_dpx"] / cu["int8x4_simd"],
                      "probe": probe}))


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "simd_rates":
        run_simd_rates(args, rank)
    elif args.workload == "serving":
        run_serving(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
