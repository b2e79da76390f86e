"""Benchmark: distance threshold search throughput on GB300.

Workload (default): the scale random-walk database -- 10,000 walks with start
times uniform in [0,200], 100..400 points, Normal(0,1) steps, starts uniform
in [0,1000]^3 (about 2.5 M entry segments resident in HBM) -- and 100 query
trajectories taken from it.  One step = one search per threshold d in
{1, 5, 15} over the full window.

value     temporal-overlap pair tests per second (pairs whose common span has
          positive length; the index-independent work of the search) of the
          headline mode (default: FP32 conservative pre-test + FP64 refine),
          with queries and results in device memory, device-timed with CUDA
          events on the stream the library launches on; the plain FP64 mode
          is measured the same way and reported beside it;
e2e       the same metric through the C ABI with host query arrays and host
          results in pinned host memory (host<->device copies inside the
          timed region);
roofline  the dominant pair kernel of each mode against its pipe's peak
          (FP64 for the plain mode, FP32 for the filter mode);
cpu_baseline / --impl reference
          the CPU FP64 oracle (time sweep, all host cores) on a bounded sample.

Multi-GPU: each rank searches its own query trajectories over its own copy of
the database (weak scaling, no collective on the data path); the timed
region is bracketed by barriers and the maximum over ranks is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1405_7461_gb300 import workloads  # noqa: E402

# Algorithmic FP64 flops per temporal-overlap pair in the plain FP64 pair
# kernel (FMA = 2): span offset 1, position of the earlier-starting segment at
# the span start 6, relative position 3, relative velocity 3, A 5, B/2 5,
# C 6, discriminant 3.
FLOPS_PER_PAIR_FP64 = 32
# Algorithmic FP32 flops per candidate pair in the filter kernel's sphere
# pre-test, written as v = E_e + K_j - 2 c_j . c_e: one add and three FMAs
# (7 flops); K_j (with the pass's bound R_j^2) is formed once per (pass of
# 128 entries, query), E_e once per entry when the index is built.
FLOPS_PER_CANDIDATE_FP32 = 7
# Peaks from unit counts and clocks (152 SMs, 2070 MHz): FP64 2 DFMA/clk/SM
# (the 1.25 TFLOP/s nominal figure), FP32 128 FFMA/clk/SM.
FP64_PEAK_GFLOPS = 2 * 2 * 152 * 2.070
FP32_PEAK_GFLOPS = 2 * 128 * 152 * 2.070
# Algorithmic DRAM bytes of the dominant kernels: the filter kernel reads each
# entry's 20 B pre-test record once per launch (the re-reads by neighbouring
# query tiles are L2/L1 hits); the plain kernel stages 64 B of every entry of
# a tile's range once per tile, i.e. 2 B per candidate pair of a full tile.
FILTER_BYTES_PER_ENTRY = 20
PLAIN_BYTES_PER_CANDIDATE = 2
# Tensor-core pre-test: the algorithmic work per pair is the rank-8 integer
# form of the sphere test (8 products accumulated, FMA = 2 flops); each MMA
# issues 128 entries x 128 query slots x 16 record elements; each entry's
# 32 B record is read from DRAM once per launch (re-reads by other
# supertiles hit L2).
FLOPS_PER_PAIR_TC = 16
TC_MMA_FLOPS = 2 * 128 * 128 * 16
TC_BYTES_PER_ENTRY = 32


def hbm_peak_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0  # fallback figure of an earlier GB300 measurement


def tensor_peak_tflops():
    """Dense FP16 tensor peak for a kernel timed alone: the measured bf16
    burst figure (FP16 and BF16 run at the same dense rate), else the
    fallback of an earlier GB300 measurement.  Returns (value, source)."""
    try:
        return (float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]),
                "MEASURED_PEAKS.json bf16_tflops, burst (of measured; FP16 dense rate = BF16)")
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback 1.9 PFLOP/s bf16 burst of an earlier GB300 measurement (of fallback)"
CPU_SAMPLE_QUERIES = 20
# The benchmark's metric (both arms report it; the value is the segment-pair
# test rate, queries/s and latencies are reported beside it).
METRIC = "segment-pair tests/s & queries/s vs plain FP64 on 1 GB300; p50/p99 query latency"
# Least wall time of the warm-up of each timed path (after its W steps).
WARMUP_MIN_S = 0.5


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fp32filter", choices=["fp32filter"],
                    help="the headline is the batched filter path; unbatched filter and plain FP64 are measured "
                         "beside it")
    ap.add_argument("--no-batching", action="store_true", help="skip the batching-workload section")
    ap.add_argument("--batch-n-traj", type=int, default=20_000)
    ap.add_argument("--batch-n-queries", type=int, default=5_000)
    ap.add_argument("--batch-oracle-queries", type=int, default=100)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-workload section")
    ap.add_argument("--serve-n-traj", type=int, default=40_000)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-plain-requests", type=int, default=400)
    ap.add_argument("--serve-oracle-requests", type=int, default=20)
    ap.add_argument("--no-self-join", action="store_true", help="skip the self-join (query (ii)) section")
    ap.add_argument("--self-join-stars", type=int, default=10_000)
    ap.add_argument("--no-tiny", action="store_true", help="skip the tiny-workload section")
    ap.add_argument("--no-precision", action="store_true", help="skip the galaxy precision-workload section")
    ap.add_argument("--galaxy-stars", type=int, default=50_000)
    ap.add_argument("--galaxy-queries", type=int, default=500)
    ap.add_argument("--galaxy-oracle-stars", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n-traj", type=int, default=10_000)
    ap.add_argument("--n-queries", type=int, default=100)
    ap.add_argument("--min-warmup-s", type=float, default=WARMUP_MIN_S,
                    help="least wall time of each timed path's warm-up (0 for profiling runs)")
    return ap.parse_args(argv)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_over_ranks(seconds, work, device="cpu"):
    """Weak-scaling reduction of one timed region: the slowest rank's time
    and the work summed over ranks (no collective outside the timing)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(work)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(w)
    return float(t.item()), float(w.item())


def workload(args, rank):
    w = workloads.scale_random_walk(n_traj=args.n_traj, n_queries=args.n_queries)
    if rank > 0:  # each rank its own query trajectories from the same database
        rng = np.random.default_rng(workloads.DEFAULT_SEED + rank)
        chosen = np.sort(rng.choice(args.n_traj, size=args.n_queries, replace=False))
        w.queries = w.entries.take(np.nonzero(np.isin(w.entries.traj_id, chosen))[0])
    return w


def config_dict(args, w, extra=None):
    c = {"workload": "scale_random_walk: %d walks (%d entry segments), %d query trajectories (%d segments), "
                     "d in {1,5,15}, full window" % (args.n_traj, len(w.entries), args.n_queries, len(w.queries)),
         "entry_segments": len(w.entries), "query_segments": len(w.queries), "d_values": list(w.d_values),
         "bin_count": 10000, "entry_chunk": HEADLINE_ENTRY_CHUNK,
         "l2": "flushed (256 MiB write) between timed GPU steps",
         "warmup_rule": "W steps, then more until %.1f s of wall time" % WARMUP_MIN_S}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def device_code_hash():
    """Hash of the library's device sources with comments and blank space
    removed: it changes when the code changes, not when a comment does."""
    import re

    csrc = os.path.join(ROOT, "paper_1405_7461_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            text = open(os.path.join(csrc, name)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            text = re.sub(r"//[^\n]*", "", text)
            h.update(name.encode())
            h.update(re.sub(r"\s+", " ", text).encode())
    return h.hexdigest()[:16]


def traffic_record(mode):
    """ncu DRAM bytes per pair-kernel launch of `mode`, if they were taken on
    the current device code (else None)."""
    path = os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")
    try:
        rec = json.load(open(path)).get(mode)
        if not rec or rec.get("device_code_sha256_16") != device_code_hash():
            return None
        return rec.get("bytes_per_launch")
    except (OSError, ValueError, AttributeError):
        return None


def cpu_baseline(w, d_values, n_sample):
    from oracle import oracle

    keep = np.unique(w.queries.traj_id)[:n_sample]
    q = w.queries.take(np.nonzero(np.isin(w.queries.traj_id, keep))[0])
    threads = oracle.default_threads()
    pairs = 0
    t = time.perf_counter()
    for d in d_values:
        r = oracle.search_sweep(w.entries, q, d, *w.window, threads=threads)
        pairs += r.overlap_pairs
    dt = time.perf_counter() - t
    # one core, on a smaller sample of the same workload (2 query trajectories, d = the first threshold)
    keep1 = keep[:2]
    q1 = w.queries.take(np.nonzero(np.isin(w.queries.traj_id, keep1))[0])
    t = time.perf_counter()
    p1 = oracle.search_sweep(w.entries, q1, d_values[0], *w.window, threads=1).overlap_pairs
    dt1 = time.perf_counter() - t
    return {"value": pairs / dt, "unit": "pair tests/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(keep)} of {w.n_query_traj} query trajectories ({len(q)} segments) x d in "
                      f"{list(d_values)}, time-sweep oracle incl. its sort, {dt:.2f} s",
            "value_1_core": p1 / dt1,
            "sample_1_core": f"{len(keep1)} query trajectories ({len(q1)} segments), d = {d_values[0]}, "
                             f"1 thread, {dt1:.2f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle

    oracle.build()
    w = workload(args, 0)
    keep = np.unique(w.queries.traj_id)[:CPU_SAMPLE_QUERIES]
    q = w.queries.take(np.nonzero(np.isin(w.queries.traj_id, keep))[0])
    threads = oracle.default_threads()

    def step():
        p = 0
        for d in w.d_values:
            p += oracle.search_sweep(w.entries, q, d, *w.window, threads=threads).overlap_pairs
        return p

    t_w = time.perf_counter()
    for _ in range(args.warmup):
        step()
    while time.perf_counter() - t_w < WARMUP_MIN_S:
        step()
    t = time.perf_counter()
    pairs = 0
    for _ in range(args.steps):
        pairs += step()
    dt = time.perf_counter() - t
    v = pairs / dt
    sample = (f"{len(keep)} of {w.n_query_traj} query trajectories ({len(q)} segments) per step x d in "
              f"{list(w.d_values)}, time-sweep oracle incl. its sort")
    line = {"impl": "reference", "metric": METRIC, "value": v,
            "unit": "pair tests/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, w, {"parallelism": "replicas" if world > 1 else "single GPU"}),
            "path": "CPU FP64 oracle (time sweep) on a bounded sample of the workload, all host cores",
            "cpu_baseline": {"value": v, "unit": "pair tests/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "pair tests/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def roofline(mode, tot, n_launch, n_entries):
    """Roofline of the dominant kernel over the timed launches: algorithmic
    work per launch / the kernel's average CUDA-event duration; beside it the
    kernel's algorithmic DRAM bytes per second against the measured HBM
    copy bandwidth."""
    kern_ms = tot["kernel_ms"] / n_launch
    if kern_ms <= 0:
        return None
    if mode == "tcfilter":
        peak, src = tensor_peak_tflops()
        sec = kern_ms / 1e3
        achieved = FLOPS_PER_PAIR_TC * tot["pairs"] / n_launch / sec / 1e12
        issued = TC_MMA_FLOPS * tot.get("mma", 0) / n_launch / sec / 1e12
        hbm_bytes = TC_BYTES_PER_ENTRY * n_entries
        gbs = hbm_bytes / sec / 1e9
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_record(mode), "kernel": "traj_dist_tc_filter_kernel", "kernel_ms_avg": kern_ms,
                "work_unit": f"{FLOPS_PER_PAIR_TC} flops per temporal-overlap pair (rank-8 integer sphere test)",
                "peak_source": src,
                "achieved_mma_issued": issued, "frac_mma_issued": issued / peak,
                "work_unit_mma_issued": "128 x 128 x 16 MACs per MMA issued (all candidates of a supertile's "
                                        "range, padded record elements included)",
                "refine_kernel_ms_avg": tot["refine_ms"] / n_launch,
                "hbm": {"algorithmic_bytes_per_launch": hbm_bytes, "achieved_gbs": gbs, "peak_gbs": hbm_peak_gbs(),
                        "frac": gbs / hbm_peak_gbs(),
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}}
    if mode == "fp64":
        work = FLOPS_PER_PAIR_FP64 * tot["fp64_pairs"] / n_launch
        peak, kernel = FP64_PEAK_GFLOPS, "traj_dist_search_kernel"
        src = "derived: 2 DFMA/clk/SM x 2 flops x 152 SMs x 2070 MHz (1.25 TFLOP/s nominal FP64)"
        per = f"{FLOPS_PER_PAIR_FP64} FP64 flops per temporal-overlap pair"
    else:
        # the unit of work is the temporal-overlap pair; the kernel tests every
        # candidate of its ranges, so the per-candidate figure is given beside it
        work = FLOPS_PER_CANDIDATE_FP32 * tot["pairs"] / n_launch
        peak, kernel = FP32_PEAK_GFLOPS, "traj_dist_filter_kernel"
        src = "derived: 128 FFMA/clk/SM x 2 flops x 152 SMs x 2070 MHz"
        per = f"{FLOPS_PER_CANDIDATE_FP32} FP32 flops per temporal-overlap pair (sphere pre-test)"
    achieved = work / (kern_ms / 1e3) / 1e9
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
         "traffic": traffic_record(mode), "kernel": kernel, "kernel_ms_avg": kern_ms, "work_unit": per,
         "peak_source": src, "clock_mhz_of_peak": 2070}
    if mode != "fp64":
        ach_c = FLOPS_PER_CANDIDATE_FP32 * tot["interactions"] / n_launch / (kern_ms / 1e3) / 1e9
        r["achieved_candidates"] = ach_c
        r["frac_candidates"] = ach_c / peak
        r["work_unit_candidates"] = f"{FLOPS_PER_CANDIDATE_FP32} FP32 flops per candidate pair of the ranges"
        r["refine_kernel_ms_avg"] = tot["refine_ms"] / n_launch
        hbm_bytes = FILTER_BYTES_PER_ENTRY * n_entries
    else:
        hbm_bytes = PLAIN_BYTES_PER_CANDIDATE * tot["interactions"] / n_launch
    gbs = hbm_bytes / (kern_ms / 1e3) / 1e9
    r["hbm"] = {"algorithmic_bytes_per_launch": hbm_bytes, "achieved_gbs": gbs, "peak_gbs": hbm_peak_gbs(),
                "frac": gbs / hbm_peak_gbs(), "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    return r


# Result capacity of the headline and end-to-end plans (4 Mi items; a step
# of the default workload returns ~2.3e4).
HEADLINE_RESULT_CAPACITY = 1 << 22


# entry chunk of the headline plan: the unit in which the pre-test's warps
# split the tiles' ranges.  On this batch (70,785 query segments, L2 flushed
# before each search) chunks of 256 / 512 / 1024 / 2048 entries gave a
# pre-test of 236 / 235 / 223 / 230 us.
HEADLINE_ENTRY_CHUNK = 1024


def headline_plan(tdq, idx, n_query_segments, host_results=False, mode=None):
    """The plan the headline (device inputs, device results) and the
    end-to-end leg (pinned host inputs read in place, results written into a
    page-locked host buffer: host_results) time: the FP32 pre-test mode (or
    `mode`), one batch of all thresholds' query segments, the default bin
    count and HEADLINE_ENTRY_CHUNK."""
    return tdq.Plan(idx, n_query_segments, mode=tdq.MODE_FP32_FILTER if mode is None else mode,
                    entry_chunk=HEADLINE_ENTRY_CHUNK, result_capacity=HEADLINE_RESULT_CAPACITY,
                    host_results=host_results)


def pinned_copy(torch, a):
    """A copy of numpy array `a` in page-locked host memory."""
    p = torch.empty(len(a), dtype=torch.from_numpy(np.asarray(a)).dtype, pin_memory=True).numpy()
    p[:] = a
    return p


def pinned_queries(tdq, torch, q, d, t0, t1):
    """The end-to-end leg's inputs: every query column, d and window in
    page-locked host memory."""
    qh = tdq.HostSegments(workloads.Segments(*[pinned_copy(torch, q[c]) for c in workloads.COLUMNS],
                                             pinned_copy(torch, q.seg_id), pinned_copy(torch, q.traj_id)))
    return qh, pinned_copy(torch, d), pinned_copy(torch, t0), pinned_copy(torch, t1)


def concat_thresholds(w):
    """The step's searches (one per threshold d) as one batch: the query set
    repeated once per d, each copy with its own segment ids and threshold."""
    k = len(w.d_values)
    q = workloads.Segments.concat([w.queries] * k)
    n = len(w.queries)
    q.seg_id = q.seg_id + np.repeat(np.arange(k, dtype=np.int64) << 40, n)
    d = np.repeat(np.asarray(w.d_values, np.float64), n)
    t0 = np.full(k * n, w.window[0])
    t1 = np.full(k * n, w.window[1])
    return q, d, t0, t1


def batching_section(args, tdq, torch, stream, with_oracle=False):
    """F2 on the batching workload: 20,000 walks x 300 points (5.98 M entries),
    5,000 fresh query trajectories of lognormal length with their own d and
    window; autotuned bin count, chunk and batch size; batches replayed as
    CUDA graphs."""
    w = workloads.batching_walks(n_traj=args.batch_n_traj, n_queries=args.batch_n_queries)
    q = w.queries
    n = len(q)
    rng = np.random.default_rng(7)
    sample_traj = rng.choice(args.batch_n_queries, size=max(1, args.batch_n_queries // 10), replace=False)
    sel = np.nonzero(np.isin(q.traj_id - 10_000_000, sample_traj))[0]
    t_tune = time.perf_counter()
    tun = tdq.autotune(w.entries, q.take(sel), w.q_d[sel], w.q_t0[sel], w.q_t1[sel], mode=tdq.MODE_FP32_FILTER,
                       stream=stream)
    tune_s = time.perf_counter() - t_tune
    idx = tdq.build_index(tdq.DeviceSegments(w.entries), bin_count=tun["bin_count"], stream=stream)
    qdev = tdq.DeviceSegments(q)
    dd, t0, t1 = (torch.from_numpy(a).cuda() for a in (w.q_d, w.q_t0, w.q_t1))
    b = int(tun["batch_query_segments"])
    plan = tdq.Plan(idx, b, mode=tdq.MODE_FP32_FILTER, entry_chunk=tun["entry_chunk"],
                    result_capacity=tun["result_capacity"])
    batches = [(a, min(a + b, n)) for a in range(0, n, b)]
    subs = [tdq.DeviceSegments(tensors=([c[a:e] for c in qdev.cols], qdev.seg_id[a:e], qdev.traj_id[a:e]))
            for a, e in batches]

    def run():
        pairs = kms = 0.0
        for (a, e), sq in zip(batches, subs):
            plan.search(sq, dd[a:e], t0[a:e], t1[a:e], stream=stream)
            st = plan.stats()
            pairs += st["overlap_pairs"]
            kms += st["pair_kernel_ms"]
        return pairs, kms

    run()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ms, pairs = [], 0.0
    for _ in range(max(1, args.steps // 2)):
        ev0.record(stream)
        p, _ = run()
        ev1.record(stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        pairs += p
    plan.free()
    # the plain FP64 path on the same batches, one step (for the batched
    # path's speedup over it)
    plan = tdq.Plan(idx, b, mode=tdq.MODE_FP64, entry_chunk=tun["entry_chunk"],
                    result_capacity=tun["result_capacity"])
    for k in {0, len(batches) - 1}:  # capture the graphs of both batch sizes before timing
        a, e = batches[k]
        plan.search(subs[k], dd[a:e], t0[a:e], t1[a:e], stream=stream)
    torch.cuda.synchronize()
    ev0.record(stream)
    p64, _ = run()
    ev1.record(stream)
    ev1.synchronize()
    ms64 = ev0.elapsed_time(ev1)
    plan.free()
    idx.free()
    tot = sum(ms) / 1e3
    out = {"workload": "batching_walks: %d walks x 300 points (%d entries), %d query trajectories (%d segments), "
                       "own d and window each" % (args.batch_n_traj, len(w.entries), args.batch_n_queries, n),
           "tuning": tun, "autotune_s": tune_s, "batches_per_step": len(batches),
           "pair_tests_per_s": pairs / tot, "queries_per_s": len(ms) * args.batch_n_queries / tot,
           "ms_per_step": 1e3 * tot / len(ms),
           "plain_fp64": {"pair_tests_per_s": p64 / (ms64 / 1e3), "queries_per_s": args.batch_n_queries / (ms64 / 1e3),
                          "ms_per_step": ms64, "steps": 1}}
    out["speedup_vs_plain_fp64"] = out["queries_per_s"] / out["plain_fp64"]["queries_per_s"]
    if with_oracle:
        from oracle import oracle

        ns = min(args.batch_oracle_queries, args.batch_n_queries)
        keep = np.random.default_rng(41).choice(args.batch_n_queries, size=ns, replace=False)
        osel = np.nonzero(np.isin(q.traj_id - 10_000_000, keep))[0]
        qs = q.take(osel)
        _, out["cpu_baseline"] = _oracle_leg(
            lambda th: oracle.search_sweep_per_query(w.entries, qs, w.q_d[osel], w.q_t0[osel], w.q_t1[osel],
                                                     threads=th),
            lambda r: r.overlap_pairs, ns,
            f"{ns} of {args.batch_n_queries} query trajectories ({len(qs)} segments, own d and window each), "
            "time-sweep oracle incl. its sort")
    return out


def self_join_section(args, tdq, torch):
    """F4, query (ii) of Sec. 2.1 with the database as the query set: the
    galaxy-disk workload's stars (200 points each) joined with themselves at
    d = 0.1 kpc over the full extent, each pair of segments of different
    stars once.  Filter mode timed over 3 runs after a warm-up; the plain FP64
    path once for comparison.  pair tests = temporal-overlap pairs of the
    ordered (query, entry) set, as for the searches."""
    w = workloads.galaxy_disk(n_stars=args.self_join_stars, n_queries=1)
    ent = w.entries
    d = 0.1
    idx = tdq.build_index(tdq.DeviceSegments(ent))
    dev = tdq.DeviceSegments(ent)
    out = {"workload": "galaxy_disk self-join: %d stars x 200 points (%d segments), d = %.2f kpc, full extent"
                       % (args.self_join_stars, len(ent), d)}
    for name, mode, reps in (("tcfilter", tdq.MODE_TC_FILTER, 3), ("fp32filter", tdq.MODE_FP32_FILTER, 3),
                             ("fp64", tdq.MODE_FP64, 1)):
        tdq.self_join(idx, dev, d, mode=mode)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            res = tdq.self_join(idx, dev, d, mode=mode)
        dt = (time.perf_counter() - t) / reps
        st = tdq.get_stats(idx)
        out[name] = {"ms": 1e3 * dt, "pair_tests_per_s": st["overlap_pairs"] / dt, "results": len(res),
                     "overlap_pairs": st["overlap_pairs"], "interactions": st["interactions"],
                     "fp64_pairs": st["fp64_pairs"]}
    out["speedup_vs_plain_fp64"] = out["fp64"]["ms"] / out["fp32filter"]["ms"]
    idx.free()
    return out


def serving_section(args, tdq, torch, with_oracle=False):
    """F3: 40,000 walks x 500 points resident (19.96 M entries); Poisson
    arrivals at 2,000/s for 10 s, each a fresh walk of 5..499 segments with
    its own d and window; p50/p99 latency and queries/s of the serving loop,
    its saturation throughput, and the plain FP64 search issued one query at
    a time for comparison."""
    import gc
    import threading

    # the sections before this one leave large host arrays behind: collect
    # them now, and keep the collector from pausing the Python client (the
    # submitter and the collecting thread) during the timed open loop
    gc.collect()
    db = workloads.serving_database(n_traj=args.serve_n_traj, n_points=500)
    reqs = workloads.serving_requests(n_requests=int(args.serve_rate * args.serve_seconds),
                                      rate_per_s=args.serve_rate, n_points=500)
    idx = tdq.build_index(tdq.DeviceSegments(db))
    del db
    srv = tdq.Server(idx, max_batch_query_segments=65536, memory_cap_bytes=16 << 30, lanes=3,
                     mode=tdq.MODE_FP32_FILTER, results_per_query_segment=1.0)
    # warm up: graph capture per size class and lane -- requests one at a
    # time, then bursts that the lanes batch into every larger class
    for rq in reqs[:50]:
        srv.wait(srv.submit(rq.query, rq.d, rq.t0, rq.t1))
    for n_burst in (8, 32, 128, 512):
        for rep in range(3):
            ws = reqs[50 + rep * n_burst:50 + (rep + 1) * n_burst]
            for t in srv.submit_many([rq.query for rq in ws], [rq.d for rq in ws], [rq.t0 for rq in ws],
                                     [rq.t1 for rq in ws]):
                srv.wait(t)
    tickets = [None] * len(reqs)
    lat = np.zeros(len(reqs))

    def submitter():
        t_start = time.perf_counter()
        for k, rq in enumerate(reqs):
            delay = rq.arrival_s - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            tickets[k] = srv.submit(rq.query, rq.d, rq.t0, rq.t1)

    gc.collect()
    gc.disable()
    t0 = time.perf_counter()
    th = threading.Thread(target=submitter)
    th.start()
    n_results = 0
    try:
        for k in range(len(reqs)):
            while tickets[k] is None:
                time.sleep(0.0002)
            res, info = srv.wait(tickets[k])
            lat[k] = info["latency_ms"]
            n_results += len(res)
        th.join()
    finally:
        gc.enable()
    wall = time.perf_counter() - t0
    st = srv.stats()
    # saturation: a burst of all requests at once from the Python client
    # (one call per request), then from one C call (the server's own ceiling)
    t1 = time.perf_counter()
    burst = [srv.submit(rq.query, rq.d, rq.t0, rq.t1) for rq in reqs]
    for t in burst:
        srv.wait(t)
    burst_s = time.perf_counter() - t1
    qs_all, d_all, a_all, b_all = [rq.query for rq in reqs], [rq.d for rq in reqs], [rq.t0 for rq in reqs], \
        [rq.t1 for rq in reqs]
    t1 = time.perf_counter()
    many = srv.submit_many(qs_all, d_all, a_all, b_all)
    srv.drain()
    many_s = time.perf_counter() - t1
    for t in many:
        srv.wait(t)
    srv.free()
    # plain FP64 search, one query at a time (host API, blocking)
    n_plain = min(len(reqs), args.serve_plain_requests)
    plat = np.zeros(n_plain)
    for rq in reqs[:5]:
        tdq.search(idx, rq.query, rq.d, rq.t0, rq.t1, mode=tdq.MODE_FP64)
    tp = time.perf_counter()
    for k, rq in enumerate(reqs[:n_plain]):
        a = time.perf_counter()
        tdq.search(idx, rq.query, rq.d, rq.t0, rq.t1, mode=tdq.MODE_FP64)
        plat[k] = 1e3 * (time.perf_counter() - a)
    plain_s = time.perf_counter() - tp
    idx.free()
    cpu = None
    if with_oracle:
        from oracle import oracle

        ns = min(args.serve_oracle_requests, len(reqs))
        picked = [reqs[k] for k in np.random.default_rng(43).choice(len(reqs), size=ns, replace=False)]
        qs = workloads.Segments.concat([rq.query for rq in picked])
        rep = [len(rq.query) for rq in picked]
        qd, q0, q1 = (np.repeat([getattr(rq, f) for rq in picked], rep) for f in ("d", "t0", "t1"))
        db = workloads.serving_database(n_traj=args.serve_n_traj, n_points=500)
        _, cpu = _oracle_leg(lambda th: oracle.search_sweep_per_query(db, qs, qd, q0, q1, threads=th),
                             lambda r: r.overlap_pairs, ns,
                             f"{ns} of {len(reqs)} requests ({len(qs)} segments, own d and window each), time-sweep "
                             "oracle incl. its sort")
        del db
    return {"cpu_baseline": cpu, "workload": "serving_walks: %d walks x 500 points resident (%d entries); Poisson arrivals %.0f/s for "
                        "%.0f s (%d requests of 5..499 segments, own d in [1,20] and window)"
                        % (args.serve_n_traj, args.serve_n_traj * 499, args.serve_rate, args.serve_seconds,
                           len(reqs)),
            "open_loop": {"queries_per_s": len(reqs) / wall, "p50_latency_ms": float(np.percentile(lat, 50)),
                          "p99_latency_ms": float(np.percentile(lat, 99)), "max_latency_ms": float(lat.max()),
                          "batches": st["batches"], "max_concurrent_batches": st["max_concurrent_batches"],
                          "results": n_results},
            "saturation_queries_per_s": len(reqs) / burst_s,
            "saturation_note": "Python client: one submit call per request, results collected per request",
            "server_saturation_queries_per_s": len(reqs) / many_s,
            "server_saturation_note": "all requests queued by one tdq_server_submit_many call (host copies "
                                      "included), timed until tdq_server_drain returns (every request searched)",
            "plain_fp64_one_at_a_time": {"queries_per_s": n_plain / plain_s,
                                         "p50_latency_ms": float(np.percentile(plat, 50)),
                                         "p99_latency_ms": float(np.percentile(plat, 99)),
                                         "sample_requests": n_plain},
            "lanes": 3, "memory_cap_bytes": 16 << 30}


def _event_time(torch, stream, fn, reps):
    """fn() run `reps` times between two CUDA events on `stream`, after one
    untimed call; returns (ms per call, last return value)."""
    out = fn()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        out = fn()
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / reps, out


def _oracle_leg(run, pairs_of, n_query_traj, sample):
    """The CPU oracle timed on a bounded sample: run() -> oracle result(s);
    pairs_of(result) -> temporal-overlap pairs."""
    from oracle import oracle

    threads = oracle.default_threads()
    t = time.perf_counter()
    res = run(threads)
    dt = time.perf_counter() - t
    pairs = pairs_of(res)
    return res, {"value": pairs / dt, "unit": "pair tests/s", "queries_per_s": n_query_traj / dt, "cores": threads,
                 "kind": "oracle", "sample": sample + f", {dt:.2f} s"}


def _compare_sample(gpu_q, gpu_e, gpu_in, gpu_out, ref, q_ids, e_ids):
    """Pair sets and endpoint differences of the GPU's results for a sample
    of query segments against the oracle's on the same sample (ids on both
    sides): pairs on one side only, and the largest relative endpoint
    difference over the matched pairs."""
    ko = q_ids[ref.query_index].astype(np.int64), e_ids[ref.entry_index].astype(np.int64)
    go = np.lexsort((gpu_e, gpu_q))
    oo = np.lexsort((ko[1], ko[0]))
    gk = np.stack([gpu_q[go], gpu_e[go]], 1)
    ok = np.stack([ko[0][oo], ko[1][oo]], 1)
    same = len(gk) == len(ok) and np.array_equal(gk, ok)
    rel = 0.0
    if same and len(gk):
        for g, o in ((gpu_in[go], ref.t_enter[oo]), (gpu_out[go], ref.t_exit[oo])):
            rel = max(rel, float(np.max(np.abs(g - o) / np.maximum(1.0, np.abs(o)))))
    only = len(set(map(tuple, gk.tolist())) ^ set(map(tuple, ok.tolist()))) if not same else 0
    return {"pairs": int(len(ok)), "pairs_on_one_side_only": int(only), "max_endpoint_rel_diff": rel}


def tiny_section(args, tdq, torch, stream, with_oracle):
    """Configuration 1: 200 random walks x 100 points (19,800 entries), 20
    query trajectories from the set (1,980 segments), d = 5, window [0, 99];
    both modes device-timed; the oracle (time sweep) over the whole query set."""
    w = workloads.tiny_random_walk()
    idx = tdq.build_index(tdq.DeviceSegments(w.entries), stream=stream)
    qdev = tdq.DeviceSegments(w.queries)
    buf = tdq.DeviceResultBuffer(1 << 16)
    d = w.d_values[0]
    out = {"workload": "tiny_random_walk: 200 walks x 100 points (%d entries), 20 query trajectories (%d segments), "
                       "d = 5, window [0, 99]" % (len(w.entries), len(w.queries))}
    for name, mode in (("tcfilter", tdq.MODE_TC_FILTER), ("fp32filter", tdq.MODE_FP32_FILTER),
                       ("fp64", tdq.MODE_FP64)):
        ms, n = _event_time(torch, stream, lambda: tdq.search_device(idx, qdev, d, *w.window, buf, stream=stream,
                                                                     mode=mode), 50)
        st = tdq.get_stats(idx)
        out[name] = {"ms_per_search": ms, "pair_tests_per_s": st["overlap_pairs"] / (ms / 1e3),
                     "queries_per_s": w.n_query_traj / (ms / 1e3), "results": n, "overlap_pairs": st["overlap_pairs"]}
    if with_oracle:
        from oracle import oracle

        _, out["cpu_baseline"] = _oracle_leg(
            lambda th: oracle.search_sweep(w.entries, w.queries, d, *w.window, threads=th),
            lambda r: r.overlap_pairs, w.n_query_traj, "all 20 query trajectories, time-sweep oracle incl. its sort")
    idx.free()
    return out


def precision_section(args, tdq, torch, stream, with_oracle):
    """Configuration 3: 50,000 disk-galaxy stars x 200 points (9.95 M
    entries), 500 query stars from the set, d in {0.01, 0.1, 1} kpc over the
    full extent; per d the filter mode and the plain FP64 path, device-timed
    on device inputs and results (the result buffer sized by a first call);
    pre-test survivors and FP64 pairs per temporal-overlap pair; the oracle on
    a seeded sample of query stars beside it, with the sample's pair set and
    endpoint difference against the GPU's."""
    w = workloads.galaxy_disk(n_stars=args.galaxy_stars, n_queries=args.galaxy_queries)
    idx = tdq.build_index(tdq.DeviceSegments(w.entries), stream=stream)
    qdev = tdq.DeviceSegments(w.queries)
    reps = max(1, min(args.steps, 3))
    rows = []
    sample_traj = np.random.default_rng(31).choice(np.unique(w.queries.traj_id), size=args.galaxy_oracle_stars,
                                                   replace=False)
    sample = w.queries.take(np.nonzero(np.isin(w.queries.traj_id, sample_traj))[0])
    for d in w.d_values:
        row = {"d": d}
        small = tdq.DeviceResultBuffer(1)
        n_res = tdq.search_device(idx, qdev, d, *w.window, small, stream=stream, allow_overflow=True,
                                  mode=tdq.MODE_TC_FILTER)
        buf = tdq.DeviceResultBuffer(max(1, n_res))
        for name, mode in (("tcfilter", tdq.MODE_TC_FILTER), ("fp32filter", tdq.MODE_FP32_FILTER),
                           ("fp64", tdq.MODE_FP64)):
            tot = {"kernel_ms": 0.0, "refine_ms": 0.0, "interactions": 0, "pairs": 0, "fp64_pairs": 0,
                   "survivors": 0, "mma": 0}

            def one():
                n = tdq.search_device(idx, qdev, d, *w.window, buf, stream=stream, mode=mode)
                st = tdq.get_stats(idx)
                tot["mma"] += st["mma_issued"]
                tot["kernel_ms"] += st["pair_kernel_ms"]
                tot["refine_ms"] += st["refine_ms"]
                tot["interactions"] += st["interactions"]
                tot["pairs"] += st["overlap_pairs"]
                tot["fp64_pairs"] += st["fp64_pairs"]
                tot["survivors"] += st["filter_survivors"]
                return n

            ms, n = _event_time(torch, stream, one, reps)
            tot = {k: v * reps / (reps + 1) for k, v in tot.items()}  # the untimed first call removed
            pairs = tot["pairs"] / reps
            row[name] = {"ms_per_search": ms, "pair_tests_per_s": pairs / (ms / 1e3),
                         "queries_per_s": w.n_query_traj / (ms / 1e3), "results": n, "overlap_pairs": pairs,
                         "candidates": tot["interactions"] / reps, "fp64_pairs": tot["fp64_pairs"] / reps,
                         "roofline": roofline(name, tot, reps, len(w.entries))}
            if name != "fp64":
                row[name]["survivors"] = tot["survivors"] / reps
                row[name]["survivors_per_overlap_pair"] = tot["survivors"] / max(1.0, tot["pairs"])
                row[name]["fp64_pairs_per_overlap_pair"] = tot["fp64_pairs"] / max(1.0, tot["pairs"])
        row["speedup_vs_plain_fp64"] = row["fp64"]["ms_per_search"] / row["fp32filter"]["ms_per_search"]
        if with_oracle:
            from oracle import oracle

            ref, row["cpu_baseline"] = _oracle_leg(
                lambda th: oracle.search_sweep(w.entries, sample, d, *w.window, threads=th),
                lambda r: r.overlap_pairs, len(sample_traj),
                f"{len(sample_traj)} of {w.n_query_traj} query stars ({len(sample)} segments), time-sweep oracle "
                "incl. its sort")
            # the filter mode's results for the sample (ids: the segments' own)
            tdq.search_device(idx, qdev, d, *w.window, buf, stream=stream, mode=tdq.MODE_FP32_FILTER)
            sel = torch.isin(buf.query_seg_id[:n_res], torch.from_numpy(sample.seg_id).cuda())
            row["error_vs_oracle"] = _compare_sample(
                buf.query_seg_id[:n_res][sel].cpu().numpy(), buf.entry_seg_id[:n_res][sel].cpu().numpy(),
                buf.t_enter[:n_res][sel].cpu().numpy(), buf.t_exit[:n_res][sel].cpu().numpy(), ref, sample.seg_id,
                w.entries.seg_id)
        rows.append(row)
        del buf, small
        torch.cuda.empty_cache()
    idx.free()
    return {"workload": "galaxy_disk: %d stars x 200 points (%d entries), %d query stars from the set (%d segments), "
                        "d in {0.01, 0.1, 1} kpc, full extent" % (args.galaxy_stars, len(w.entries), w.n_query_traj,
                                                                 len(w.queries)),
            "per_d": rows}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_1405_7461_gb300 import build, tdq

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        torch.cuda.set_device(local)
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    build.build()
    tdq.load()
    modes = {"fp64": tdq.MODE_FP64, "fp32filter": tdq.MODE_FP32_FILTER}

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    w = workload(args, rank)
    stream = torch.cuda.current_stream()
    ent_dev = tdq.DeviceSegments(w.entries)
    idx = tdq.build_index(ent_dev, stream=stream)
    torch.cuda.synchronize()
    t_build = time.perf_counter()
    tdq.build_index(ent_dev, stream=stream).free()
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t_build
    del ent_dev
    qdev = tdq.DeviceSegments(w.queries)
    buf = tdq.DeviceResultBuffer(1 << 22)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # the batched form of a step: all thresholds in one batch (one graph launch)
    q3, d3, t03, t13 = concat_thresholds(w)
    q3dev = tdq.DeviceSegments(q3)
    d3dev, t03dev, t13dev = (torch.from_numpy(a).cuda() for a in (d3, t03, t13))
    plan = headline_plan(tdq, idx, len(q3))
    plantc = headline_plan(tdq, idx, len(q3), mode=tdq.MODE_TC_FILTER)
    modes["tcfilter"] = tdq.MODE_TC_FILTER

    def step(mode):
        # the step's searches; returns the bookkeeping to run once the step's
        # end is recorded (a batched step's statistics are read afterwards;
        # unbatched searches share the index's statistics, read after each)
        t = {"pairs": 0, "interactions": 0, "results": 0, "launches": 0, "kernel_ms": 0.0, "fp64_pairs": 0,
             "survivors": 0, "refine_ms": 0.0, "mma": 0}
        if mode in ("batched", "batched_tc"):
            p = plan if mode == "batched" else plantc
            t["results"] = p.search(q3dev, d3dev, t03dev, t13dev, stream=stream)
            return lambda: tally(t, [p.stats()])
        stats = []
        for d in w.d_values:
            t["results"] += tdq.search_device(idx, qdev, d, *w.window, buf, stream=stream, mode=modes[mode])
            stats.append(tdq.get_stats(idx))
        return lambda: tally(t, stats)

    def tally(t, stats):
        for s in stats:
            t["pairs"] += s["overlap_pairs"]
            t["interactions"] += s["interactions"]
            t["fp64_pairs"] += s["fp64_pairs"]
            t["survivors"] += s["filter_survivors"]
            t["launches"] += s["kernel_launches"]
            t["kernel_ms"] += s["pair_kernel_ms"]
            t["refine_ms"] += s["refine_ms"]
            t["mma"] += s["mma_issued"]
        return t

    def timed(mode):
        # W warm-up steps, then more until WARMUP_MIN_S of wall time has passed:
        # a few sub-millisecond steps do not bring the GPU to its steady clocks
        t_w = time.perf_counter()
        for _ in range(args.warmup):
            step(mode)()
        while time.perf_counter() - t_w < args.min_warmup_s:
            step(mode)()
        torch.cuda.synchronize()
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ms, tot = [], None
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            collect = step(mode)
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
            out = collect()
            tot = out if tot is None else {k: tot[k] + out[k] for k in tot}
        torch.cuda.synchronize()
        barrier()
        total_ms, pairs = reduce_over_ranks(sum(ms), float(tot["pairs"]), device="cuda")
        batched = mode in ("batched", "batched_tc")
        n_launch = args.steps * (1 if batched else len(w.d_values))
        kmode = {"batched": "fp32filter", "batched_tc": "tcfilter"}.get(mode, mode)
        return {"value": pairs / (total_ms / 1e3), "ms_per_step": total_ms / args.steps,
                "queries_per_s": world * args.steps * len(w.d_values) * args.n_queries / (total_ms / 1e3),
                "interactions_per_s": world * tot["interactions"] / (total_ms / 1e3),
                "fp64_pairs_per_step": tot["fp64_pairs"] / args.steps,
                "filter_survivors_per_step": tot["survivors"] / args.steps,
                "results_per_step": tot["results"] / args.steps, "gpu_launches": int(tot["launches"]),
                "roofline": roofline(kmode, tot, n_launch, len(w.entries))}

    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    head = timed("batched")
    headtc = timed("batched_tc")
    unb_tc = timed("tcfilter")
    unb = timed("fp32filter")
    plain = timed("fp64")
    clk = clocks.stop()

    # end to end through the C ABI: host queries in, host results out, both
    # in pinned host memory
    e2e = None
    if not args.no_e2e:
        q3h, d3h, t03h, t13h = pinned_queries(tdq, torch, q3, d3, t03, t13)
        # the kernels read the pinned inputs and write the results into the
        # plan's page-locked host buffer over the CPU-GPU link
        eplan = headline_plan(tdq, idx, len(q3), host_results=True)
        t_w = time.perf_counter()
        for _ in range(max(args.warmup, 1)):
            eplan.search(q3h, d3h, t03h, t13h, stream=stream)
            eplan.results(view=True)
        while time.perf_counter() - t_w < args.min_warmup_s:
            eplan.search(q3h, d3h, t03h, t13h, stream=stream)
            eplan.results(view=True)
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        d2h = 0
        for _ in range(args.steps):
            eplan.search(q3h, d3h, t03h, t13h, stream=stream)
            r = eplan.results(view=True)
            d2h += 32 * len(r) + 64
        torch.cuda.synchronize()
        e_dt = time.perf_counter() - t
        # (every step searches the same batch: the last one's count of pairs)
        e_pairs = args.steps * eplan.stats()["overlap_pairs"]
        e_dt, e_pairs = reduce_over_ranks(e_dt, e_pairs, device="cuda")
        eplan.free()
        e2e = {"value": e_pairs / e_dt, "unit": "pair tests/s", "host_memory": "pinned",
               "h2d_bytes_per_step": len(q3) * 96, "d2h_bytes_per_step": d2h // args.steps,
               "path": "pinned host queries read in place by the kernels; results written by the kernels into a "
                       "page-locked host buffer (tdq_plan host_results), read there; counters through mapped memory",
               "queries_per_s": world * args.steps * len(w.d_values) * args.n_queries / e_dt}
        # the same step through the plain host call tdq_search (the boundary's
        # search: one call per threshold, host queries in, library-owned host
        # results out), as a caller without plans makes it
        qh1 = tdq.HostSegments(workloads.Segments(*[pinned_copy(torch, w.queries[c]) for c in workloads.COLUMNS],
                                                  pinned_copy(torch, w.queries.seg_id),
                                                  pinned_copy(torch, w.queries.traj_id)))
        def host_step():
            n_pairs, n_res = 0, 0
            for d in w.d_values:
                r = tdq.search(idx, qh1, d, *w.window, mode=tdq.MODE_FP32_FILTER)
                n_pairs += tdq.get_stats(idx)["overlap_pairs"]
                n_res += len(r)
                del r
            return n_pairs, n_res
        t_w = time.perf_counter()
        for _ in range(max(args.warmup, 1)):
            host_step()
        while time.perf_counter() - t_w < args.min_warmup_s:
            host_step()
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        h_pairs = h_res = 0
        for _ in range(args.steps):
            p_, r_ = host_step()
            h_pairs += p_
            h_res += r_
        torch.cuda.synchronize()
        h_dt, h_pairs = reduce_over_ranks(time.perf_counter() - t, h_pairs, device="cuda")
        e2e["tdq_search"] = {
            "value": h_pairs / h_dt, "unit": "pair tests/s", "host_memory": "pinned",
            "h2d_bytes_per_step": len(w.queries) * 80 * len(w.d_values),
            "d2h_bytes_per_step": 32 * h_res // args.steps,
            "path": "tdq_search per threshold (FP32 pre-test mode): pinned host queries read in place, results "
                    "copied into library-owned page-locked host arrays (tdq_results), one call after another",
            "queries_per_s": world * args.steps * len(w.d_values) * args.n_queries / h_dt}

    with_oracle = not args.no_cpu_baseline
    # the latency measurement first, before the sections that leave large
    # host and device allocations behind
    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        serving = serving_section(args, tdq, torch, with_oracle)
    tiny = None
    if rank == 0 and world == 1 and not args.no_tiny:
        tiny = tiny_section(args, tdq, torch, stream, with_oracle)
    precision = None
    if rank == 0 and world == 1 and not args.no_precision:
        precision = precision_section(args, tdq, torch, stream, with_oracle)
    batching = None
    if rank == 0 and world == 1 and not args.no_batching:
        batching = batching_section(args, tdq, torch, stream, with_oracle)
    self_join = None
    if rank == 0 and world == 1 and not args.no_self_join:
        self_join = self_join_section(args, tdq, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, w.d_values, CPU_SAMPLE_QUERIES)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": head["value"], "unit": "pair tests/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, w, {"parallelism": "replicas" if world > 1 else "single GPU"}),
            "path": "FP32 conservative pre-test + FP64 refine; the three thresholds of a step batched in one "
                    "plan (one CUDA-graph launch)",
            "index_build_s": build_s,
            "queries_per_s": head["queries_per_s"],
            "interactions_per_s": head["interactions_per_s"],
            "fp64_pairs_per_step": head["fp64_pairs_per_step"],
            "filter_survivors_per_step": head["filter_survivors_per_step"],
            "results_per_step": head["results_per_step"],
            "roofline": head["roofline"],
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": head["gpu_launches"],
            "batched_tcfilter": {k: headtc[k] for k in ("value", "ms_per_step", "queries_per_s", "roofline",
                                                        "gpu_launches", "filter_survivors_per_step")},
            "unbatched_tcfilter": {k: unb_tc[k] for k in ("value", "ms_per_step", "queries_per_s", "roofline",
                                                          "gpu_launches")},
            "unbatched_fp32filter": {k: unb[k] for k in ("value", "ms_per_step", "queries_per_s", "roofline",
                                                         "gpu_launches")},
            "plain_fp64": {k: plain[k] for k in ("value", "ms_per_step", "queries_per_s", "roofline",
                                                 "gpu_launches")},
            "speedup_vs_plain_fp64": {"pair_tests": head["value"] / plain["value"],
                                      "queries": head["queries_per_s"] / plain["queries_per_s"]},
            "tiny_workload": tiny,
            "precision_workload": precision,
            "batching_workload": batching,
            "serving_workload": serving,
            "self_join_workload": self_join,
        }
        print(json.dumps(line), flush=True)
    plan.free()
    plantc.free()
    idx.free()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
