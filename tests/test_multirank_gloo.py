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
