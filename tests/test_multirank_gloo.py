"""The benchmark's multi-rank path on CPU: two gloo ranks take their own
query trajectories from the same database (weak scaling) and the timed
region reduces to the slowest rank's time and the summed work."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        class Args:
            n_traj = 300
            n_queries = 5

        w = bench.workload(Args, rank)
        secs, work = bench.reduce_over_ranks(0.5 + rank, 100.0 * (rank + 1))
        out[rank] = (len(w.entries), sorted(set(w.queries.traj_id.tolist())), secs, work, bench.dist_env())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    n0, q0, s0, w0, env0 = out[0]
    n1, q1, s1, w1, env1 = out[1]
    assert n0 == n1  # the same database on every rank
    assert q0 != q1 and len(q0) == len(q1) == 5  # each rank its own query trajectories
    assert s0 == s1 == pytest.approx(1.5)  # the slowest rank's time
    assert w0 == w1 == pytest.approx(300.0)  # work summed over ranks
    assert env0 == (0, 2, 0) and env1 == (1, 2, 1)


def test_single_process_reduction_is_identity():
    import bench

    assert bench.reduce_over_ranks(2.0, 7.0) == (2.0, 7.0)
    assert np.isfinite(bench.FP64_PEAK_GFLOPS) and bench.FP64_PEAK_GFLOPS == pytest.approx(1258.56)


def test_reference_arm_prints_the_contract_line():
    # bench.py --impl reference times the CPU oracle and prints one JSON line
    # with the fields both arms share (a reduced workload keeps this quick)
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                          "--n-traj", "1500", "--n-queries", "10"], cwd=root, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "pair tests/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("scale_random_walk")


def test_roofline_arithmetic():
    # the bench line's roofline object: algorithmic work per launch over the
    # kernel's average event time, against the derived peaks; algorithmic
    # DRAM bytes beside it
    import bench

    tot = {"kernel_ms": 2.0, "fp64_pairs": 1e9, "interactions": 4e9, "refine_ms": 0.5, "pairs": 3e9}
    r = bench.roofline("fp64", tot, 2, 1000)
    assert r["kernel_ms_avg"] == 1.0
    assert r["achieved"] == pytest.approx(32 * 0.5e9 / 1e-3 / 1e9)  # 32 flops per overlap pair, GFLOP/s
    assert r["frac"] == pytest.approx(r["achieved"] / 1258.56)
    assert r["hbm"]["algorithmic_bytes_per_launch"] == pytest.approx(2 * 2e9)  # 2 B per candidate
    f = bench.roofline("fp32filter", tot, 2, 1000)
    assert f["achieved"] == pytest.approx(7 * 1.5e9 / 1e-3 / 1e9)  # 7 flops per temporal-overlap pair
    assert f["frac"] == pytest.approx(f["achieved"] / 80547.84)
    assert f["achieved_candidates"] == pytest.approx(7 * 2e9 / 1e-3 / 1e9)  # 7 flops per candidate
    assert f["frac_candidates"] == pytest.approx(f["achieved_candidates"] / 80547.84)
    assert f["refine_kernel_ms_avg"] == 0.25
    assert f["hbm"]["algorithmic_bytes_per_launch"] == 20 * 1000  # the 20 B record of each entry
    assert f["hbm"]["frac"] == pytest.approx(f["hbm"]["achieved_gbs"] / bench.hbm_peak_gbs())
    assert bench.roofline("fp64", dict(tot, kernel_ms=0.0), 2, 1000) is None
    # the tensor-core pre-test: 16 flops (the rank-8 integer form) per
    # temporal-overlap pair against the dense tensor peak; the MMAs issued
    # (128 x 128 x 16 MACs each) beside it; 32 B record per entry from DRAM
    t = bench.roofline("tcfilter", dict(tot, mma=1000), 2, 1000)
    peak, _ = bench.tensor_peak_tflops()
    assert t["bound"] == "tensor" and t["unit"] == "TFLOP/s"
    assert t["achieved"] == pytest.approx(16 * 1.5e9 / 1e-3 / 1e12)
    assert t["frac"] == pytest.approx(t["achieved"] / peak)
    assert t["achieved_mma_issued"] == pytest.approx(2 * 128 * 128 * 16 * 500 / 1e-3 / 1e12)
    assert t["hbm"]["algorithmic_bytes_per_launch"] == 32 * 1000
