"""Benchmark: distance threshold search throughput on GB300.

Workload (default): the scale random-walk database -- 10,000 walks with start
times uniform in [0,200], 100..400 points, Normal(0,1) steps, starts uniform
in [0,1000]^3 (about 2.5 M entry segments resident in HBM) -- and 100 query
trajectories taken from it.  One step = one search per threshold d in
{1, 5, 15} over the full window.

value     temporal-overlap pair tests per second (pairs whose common span has
          positive length; the index-independent work of the search), with
          queries and results in device memory, device-timed with CUDA events
          on the stream the library launches on;
e2e       the same metric through the C ABI with host query arrays and host
          results (host<->device copies inside the timed region);
roofline  the pair kernel (the dominant kernel) against the FP64 issue peak;
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
# FP64 peak from the unit counts and clocks: 2 DFMA per clock per SM x 2
# flops x 152 SMs x 2070 MHz (the 1.25 TFLOP/s nominal figure).
FP64_PEAK_GFLOPS = 2 * 2 * 152 * 2.070
CPU_SAMPLE_QUERIES = 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fp64", choices=["fp64", "fp32filter"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n-traj", type=int, default=10_000)
    ap.add_argument("--n-queries", type=int, default=100)
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


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
         "bin_count": 10000, "mode": args.mode, "l2": "flushed (256 MiB write) between timed steps"}
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


def traffic_record():
    """ncu DRAM bytes per pair-kernel launch, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_1405_7461_gb300", "csrc", "search.cu")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if rec.get("search_cu_sha256_16") != h or rec.get("mode") is None:
            return None
        return rec
    except (OSError, ValueError):
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
    return {"value": pairs / dt, "unit": "pair tests/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(keep)} of {w.n_query_traj} query trajectories ({len(q)} segments) x d in "
                      f"{list(d_values)}, time-sweep oracle incl. its sort, {dt:.2f} s"}


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

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    pairs = 0
    for _ in range(args.steps):
        pairs += step()
    dt = time.perf_counter() - t
    v = pairs / dt
    sample = (f"{len(keep)} of {w.n_query_traj} query trajectories ({len(q)} segments) per step x d in "
              f"{list(w.d_values)}, time-sweep oracle incl. its sort")
    line = {"impl": "reference", "metric": "segment-pair tests/s (temporal-overlap pairs)", "value": v,
            "unit": "pair tests/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config_dict(args, w, {"sample": sample}),
            "cpu_baseline": {"value": v, "unit": "pair tests/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "pair tests/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
    mode = tdq.MODE_FP64 if args.mode == "fp64" else tdq.MODE_FP32_FILTER

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    w = workload(args, rank)
    stream = torch.cuda.current_stream()
    ent_dev = tdq.DeviceSegments(w.entries)
    idx = tdq.build_index(ent_dev, stream=stream)
    t_build = time.perf_counter()
    tdq.build_index(ent_dev, stream=stream).free()
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t_build
    del ent_dev
    qdev = tdq.DeviceSegments(w.queries)
    cap = 1 << 22
    buf = tdq.DeviceResultBuffer(cap)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        pairs = inter = res = launches = 0
        kms = 0.0
        for d in w.d_values:
            cnt = tdq.search_device(idx, qdev, d, *w.window, buf, stream=stream, mode=mode)
            s = tdq.get_stats(idx)
            pairs += s["overlap_pairs"]
            inter += s["interactions"]
            res += cnt
            launches += s["kernel_launches"]
            kms += s["pair_kernel_ms"]
        return pairs, inter, res, launches, kms

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ms, tot = [], [0, 0, 0, 0, 0.0]
    for _ in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        out = step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        for k in range(5):
            tot[k] += out[k]
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
        p = torch.tensor([float(tot[0])], device="cuda")
        torch.distributed.all_reduce(p)
        all_pairs = float(p.item())
    else:
        all_pairs = float(tot[0])
    value = all_pairs / (total_ms / 1e3)
    queries_per_s = world * args.steps * len(w.d_values) * args.n_queries / (total_ms / 1e3)
    n_pair_launches = args.steps * len(w.d_values)
    kern_ms = tot[4] / n_pair_launches
    flops_per_launch = FLOPS_PER_PAIR_FP64 * tot[0] / n_pair_launches
    achieved = flops_per_launch / (kern_ms / 1e3) / 1e9
    trec = traffic_record()
    traffic = None
    if trec and trec.get("mode") == args.mode:
        traffic = trec.get("bytes_per_launch")

    # end to end through the C ABI: host queries in, host results out
    e2e = None
    if not args.no_e2e:
        qhost = tdq.HostSegments(w.queries)
        tdq.search(idx, qhost, w.d_values[0], *w.window, stream=stream, mode=mode)
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        e_pairs = 0
        d2h = 0
        for _ in range(args.steps):
            for d in w.d_values:
                r = tdq.search(idx, qhost, d, *w.window, stream=stream, mode=mode)
                e_pairs += tdq.get_stats(idx)["overlap_pairs"]
                d2h += 32 * len(r) + 64
        torch.cuda.synchronize()
        e_dt = time.perf_counter() - t
        if world > 1:
            tt = torch.tensor([e_dt], device="cuda")
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            e_dt = float(tt.item())
        e2e = {"value": world * e_pairs / e_dt, "unit": "pair tests/s",
               "h2d_bytes_per_step": len(w.d_values) * len(w.queries) * 72,
               "d2h_bytes_per_step": d2h // args.steps,
               "queries_per_s": world * args.steps * len(w.d_values) * args.n_queries / e_dt}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, w.d_values, CPU_SAMPLE_QUERIES)

    if rank == 0:
        line = {
            "metric": "segment-pair tests/s (temporal-overlap pairs), plain FP64 search" if args.mode == "fp64"
            else "segment-pair tests/s (temporal-overlap pairs), FP32 filter + FP64 refine",
            "value": value, "unit": "pair tests/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, w, {"parallelism": "replicas" if world > 1 else "single GPU",
                                            "index_build_s": build_s}),
            "queries_per_s": queries_per_s,
            "interactions_per_s": world * tot[1] / (total_ms / 1e3),
            "results_per_step": tot[2] / args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic,
                         "kernel": "traj_dist_search_kernel", "kernel_ms_avg": kern_ms,
                         "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (1.25 TFLOP/s nominal FP64)"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": int(tot[3]),
        }
        print(json.dumps(line), flush=True)
    idx.free()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
