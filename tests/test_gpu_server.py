"""Serving loop: continuous batching gives every request the same results
alone and in the mix, matches the oracle, honours the memory cap, and
reports timeouts and invalid requests on the host."""
import threading

import numpy as np
import pytest

from oracle import oracle
from paper_1405_7461_gb300 import workloads
from tests._util import compare_results

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tdq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7461_gb300 import build, tdq as t

    build.build()
    t.load()
    return t


@pytest.fixture(scope="module")
def db():
    return workloads.serving_database(n_traj=3000, n_points=120)


@pytest.fixture(scope="module")
def requests():
    return workloads.serving_requests(n_requests=48, rate_per_s=2000.0, n_points=120, min_seg=5, max_seg=110)


def _sorted(r):
    o = np.lexsort((r.entry_seg_id, r.query_seg_id))
    return r.query_seg_id[o], r.entry_seg_id[o], r.t_enter[o], r.t_exit[o]


def _same(a, b):
    for x, y in zip(_sorted(a), _sorted(b)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("mode_name", ["filter", "tcfilter", "fp64"])
def test_results_same_alone_and_in_the_mix(tdq, db, requests, mode_name):
    mode = {"fp64": tdq.MODE_FP64, "filter": tdq.MODE_FP32_FILTER, "tcfilter": tdq.MODE_TC_FILTER}[mode_name]
    with tdq.build_index(db) as idx:
        with tdq.Server(idx, max_batch_query_segments=2048, lanes=3, mode=mode) as srv:
            alone = []
            for rq in requests:
                res, info = srv.wait(srv.submit(rq.query, rq.d, rq.t0, rq.t1))
                alone.append(res)
                assert info["latency_ms"] >= info["run_ms"] >= 0
            st_alone = srv.stats()
            assert st_alone["batches"] == len(requests)
            # the mix, 1: all requests queued in one call, so that the lanes
            # admit several into each batch
            tickets = srv.submit_many([rq.query for rq in requests], [rq.d for rq in requests],
                                      [rq.t0 for rq in requests], [rq.t1 for rq in requests])
            mixed = [srv.wait(t)[0] for t in tickets]
            st_many = srv.stats()
            assert st_many["batches"] - st_alone["batches"] < len(requests)  # requests shared batches
            # the mix, 2: all requests submitted from two threads at once (they
            # share batches or not, as the timing falls)
            tickets = [None] * len(requests)

            def submitter(ks):
                for k in ks:
                    rq = requests[k]
                    tickets[k] = srv.submit(rq.query, rq.d, rq.t0, rq.t1)

            ths = [threading.Thread(target=submitter, args=(range(i, len(requests), 2),)) for i in range(2)]
            for t in ths:
                t.start()
            for t in ths:
                t.join()
            mixed2 = [srv.wait(t)[0] for t in tickets]
            st = srv.stats()
        assert st["requests_completed"] == 3 * len(requests)
        for a, m, m2 in zip(alone, mixed, mixed2):
            _same(a, m)
            _same(a, m2)
        # each request against a direct search with its own d and window
        for rq, a in zip(requests[:8], alone[:8]):
            ref = tdq.search(idx, rq.query, rq.d, rq.t0, rq.t1)
            _same(a, ref)
    assert sum(len(a) for a in alone) > 0


def test_request_results_match_the_oracle(tdq, db, requests):
    with tdq.build_index(db) as idx, tdq.Server(idx, lanes=2) as srv:
        tickets = [srv.submit(rq.query, rq.d, rq.t0, rq.t1) for rq in requests[:12]]
        got = [srv.wait(t)[0] for t in tickets]
    matched = 0
    for rq, g in zip(requests[:12], got):
        ref = oracle.search_sweep(db, rq.query, rq.d, rq.t0, rq.t1)
        qpos = {int(s): i for i, s in enumerate(rq.query.seg_id)}
        gi = {"qi": np.array([qpos[int(s)] for s in g.query_seg_id], np.int64), "ei": g.entry_seg_id.copy(),
              "t_enter": g.t_enter, "t_exit": g.t_exit}
        cmp = compare_results(gi, {"qi": ref.query_index, "ei": ref.entry_index, "t_enter": ref.t_enter,
                                   "t_exit": ref.t_exit}, db, rq.query, rq.d, rq.t0, rq.t1,
                              dmin_fn=lambda ei, qi: oracle.pair_dmin(db, ei, rq.query, qi, rq.t0, rq.t1))
        matched += cmp["matched"]
    assert matched > 0


def test_memory_cap_admits_one_request_at_a_time(tdq, db, requests):
    with tdq.build_index(db) as idx:
        with tdq.Server(idx, lanes=3, memory_cap_bytes=1) as srv:
            tickets = [srv.submit(rq.query, rq.d, rq.t0, rq.t1) for rq in requests[:20]]
            got = [srv.wait(t)[0] for t in tickets]
            st = srv.stats()
        assert st["batches"] == 20 and st["max_concurrent_batches"] == 1
        for rq, g in zip(requests[:20], got):
            _same(g, tdq.search(idx, rq.query, rq.d, rq.t0, rq.t1))


def test_submit_many_equals_one_by_one_and_is_all_or_nothing(tdq, db, requests):
    """tdq_server_submit_many queues many requests in one call: each
    request's results equal those of its own submit; a batch holding one
    invalid request queues nothing; tdq_server_drain returns once every
    request has been searched."""
    rq = requests[:24]
    with tdq.build_index(db) as idx, tdq.Server(idx, lanes=2) as srv:
        one = [srv.wait(srv.submit(r.query, r.d, r.t0, r.t1))[0] for r in rq]
        tickets = srv.submit_many([r.query for r in rq], [r.d for r in rq], [r.t0 for r in rq], [r.t1 for r in rq])
        srv.drain()
        st = srv.stats()
        assert st["requests_completed"] == 2 * len(rq) and st["queued"] == 0
        many = [srv.wait(t, 0)[0] for t in tickets]  # done already: no waiting
        bad_d = [r.d for r in rq]
        bad_d[5] = -1.0
        before = srv.stats()["requests_submitted"]
        with pytest.raises(tdq.TdqError) as ei:
            srv.submit_many([r.query for r in rq], bad_d, [r.t0 for r in rq], [r.t1 for r in rq])
        assert ei.value.status == tdq.TDQ_ERR_INVALID and "request 5" in str(ei.value)
        assert srv.stats()["requests_submitted"] == before
    assert sum(len(a) for a in one) > 0
    for a, b in zip(one, many):
        _same(a, b)


def test_timeouts_and_invalid_requests_are_reported_on_the_host(tdq, db, requests):
    with tdq.build_index(db) as idx, tdq.Server(idx, lanes=1, max_batch_query_segments=512) as srv:
        rq = requests[0]
        with pytest.raises(tdq.TdqError) as ei:
            srv.submit(rq.query, -1.0, rq.t0, rq.t1)
        assert ei.value.status == tdq.TDQ_ERR_INVALID
        with pytest.raises(tdq.TdqError) as ei:
            srv.submit(rq.query, rq.d, 5.0, 1.0)
        assert ei.value.status == tdq.TDQ_ERR_INVALID
        big = workloads.Segments.concat([requests[k].query for k in range(12)])
        if len(big) > 512:
            with pytest.raises(tdq.TdqError):
                srv.submit(big, 1.0, -np.inf, np.inf)
        with pytest.raises(tdq.TdqError) as ei:
            srv.wait(987654321, 0)
        assert ei.value.status == tdq.TDQ_ERR_INVALID
        # a wait that runs out of time leaves the request waitable
        tickets = [srv.submit(r.query, r.d, r.t0, r.t1) for r in requests[:10]]
        try:
            srv.wait(tickets[-1], 0)
        except tdq.TdqError as e:
            assert e.status == tdq.TDQ_ERR_TIMEOUT
        for t in tickets:
            srv.wait(t)


def test_serving_workload_full_size_sampled(tdq):
    """The serving workload at full size: 40,000 walks x 500 points (19.96 M
    entries) resident, the benchmark's server settings (3 lanes, 16 GiB cap,
    batches up to 65,536 segments, filter mode); 64 requests submitted at
    once; a seeded sample of 4 is checked pair by pair against the oracle."""
    db = workloads.serving_database(n_traj=40_000, n_points=500)
    reqs = workloads.serving_requests(n_requests=64, rate_per_s=2000.0, n_points=500)
    with tdq.build_index(tdq.DeviceSegments(db)) as idx, \
            tdq.Server(idx, max_batch_query_segments=65536, memory_cap_bytes=16 << 30, lanes=3,
                       mode=tdq.MODE_FP32_FILTER, results_per_query_segment=1.0) as srv:
        tickets = [srv.submit(rq.query, rq.d, rq.t0, rq.t1) for rq in reqs]
        got = [srv.wait(t)[0] for t in tickets]
    matched = 0
    for k in np.random.default_rng(3).choice(len(reqs), size=4, replace=False):
        rq, g = reqs[k], got[k]
        ref = oracle.search_sweep(db, rq.query, rq.d, rq.t0, rq.t1)
        qpos = {int(s): i for i, s in enumerate(rq.query.seg_id)}
        gi = {"qi": np.array([qpos[int(s)] for s in g.query_seg_id], np.int64), "ei": g.entry_seg_id.copy(),
              "t_enter": g.t_enter, "t_exit": g.t_exit}
        cmp = compare_results(gi, {"qi": ref.query_index, "ei": ref.entry_index, "t_enter": ref.t_enter,
                                   "t_exit": ref.t_exit}, db, rq.query, rq.d, rq.t0, rq.t1,
                              dmin_fn=lambda ei, qi: oracle.pair_dmin(db, ei, rq.query, qi, rq.t0, rq.t1))
        assert cmp["matched"] == len(ref.query_index)
        matched += cmp["matched"]
    assert matched > 0
