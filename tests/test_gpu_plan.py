"""Batched plans (one CUDA graph launch per batch) and the autotuner, against
the oracle and against the unbatched device search."""
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


def _positions(ids, pool):
    order = np.argsort(pool, kind="stable")
    pos = np.searchsorted(pool[order], ids)
    assert np.all(pool[order][pos] == ids)
    return order[pos]


def _key_sorted(r):
    o = np.lexsort((r.entry_seg_id, r.query_seg_id))
    return r.query_seg_id[o], r.entry_seg_id[o], r.t_enter[o], r.t_exit[o]


def _same(a, b):
    for x, y in zip(_key_sorted(a), _key_sorted(b)):
        assert np.array_equal(x, y)


def _oracle_per_trajectory(w, q, qd, q0, q1):
    parts = {k: [] for k in ("qi", "ei", "t_enter", "t_exit")}
    for tj in np.unique(q.traj_id):
        sel = np.nonzero(q.traj_id == tj)[0]
        r = oracle.search_sweep(w.entries, q.take(sel), qd[sel[0]], q0[sel[0]], q1[sel[0]])
        parts["qi"].append(sel[r.query_index])
        parts["ei"].append(r.entry_index)
        parts["t_enter"].append(r.t_enter)
        parts["t_exit"].append(r.t_exit)
    return {k: np.concatenate(v) for k, v in parts.items()}


@pytest.mark.parametrize("mode_name", ["fp64", "filter", "tcfilter"])
def test_plan_batches_match_oracle_and_unbatched_search(tdq, mode_name):
    mode = {"fp64": tdq.MODE_FP64, "filter": tdq.MODE_FP32_FILTER, "tcfilter": tdq.MODE_TC_FILTER}[mode_name]
    w = workloads.batching_walks(n_traj=500, n_queries=80, box=50.0)
    q = w.queries
    n = len(q)
    with tdq.build_index(w.entries, bin_count=3000) as idx:
        # reference: the unbatched device search with per-query parameters
        buf = tdq.DeviceResultBuffer(1 << 18)
        cnt = tdq.search_device_batched(idx, tdq.DeviceSegments(q), torch.from_numpy(w.q_d).cuda(),
                                        torch.from_numpy(w.q_t0).cuda(), torch.from_numpy(w.q_t1).cuda(), buf,
                                        mode=mode)
        ref = buf.to_host(cnt)
        ref_overlap = tdq.get_stats(idx)["overlap_pairs"]
        # the same queries as uneven batches through one plan (graph replay,
        # several size classes, so most batches carry padding slots); host
        # and device inputs
        cuts = [0, 7, 1500, 1501, 4000, n]
        with tdq.Plan(idx, max_query_segments=4000, mode=mode) as plan:
            got = []
            overlap = 0
            for k, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
                if b <= a:
                    continue
                sub = q.take(np.arange(a, b))
                src = tdq.DeviceSegments(sub) if k % 2 else sub
                c = plan.search(src, w.q_d[a:b], w.q_t0[a:b], w.q_t1[a:b])
                r = plan.results()
                st = plan.stats()
                assert len(r) == c == st["results"]
                overlap += st["overlap_pairs"]
                got.append(r)
        # the overlap count is exact integer work: batching does not change it
        assert overlap == ref_overlap
        merged = tdq.Results(*[np.concatenate([getattr(r, f) for r in got])
                               for f in ("query_seg_id", "entry_seg_id", "t_enter", "t_exit")])
    _same(merged, ref)
    # against the oracle, trajectory by trajectory (own d and window each)
    ora = _oracle_per_trajectory(w, q, w.q_d, w.q_t0, w.q_t1)
    gi = {"qi": _positions(merged.query_seg_id, q.seg_id), "ei": _positions(merged.entry_seg_id, w.entries.seg_id),
          "t_enter": merged.t_enter, "t_exit": merged.t_exit}
    dmin = lambda ei, qi: oracle.pair_dmin(w.entries, ei, q, qi, w.q_t0[qi], w.q_t1[qi])  # noqa: E731
    cmp = compare_results(gi, ora, w.entries, q, None, dmin_fn=dmin, d_per_query=w.q_d,
                          win_per_query=(w.q_t0, w.q_t1))
    assert cmp["matched"] > 1000


def test_plan_graph_equals_direct_launches_and_regrows(tdq):
    """Graph replay and direct launches give identical results; a result
    buffer that is too small is grown and the batch re-run."""
    w = workloads.scale_random_walk(n_traj=1500, n_queries=12)
    q = w.queries
    n = len(q)
    d = np.full(n, 15.0)
    t0 = np.full(n, w.window[0])
    t1 = np.full(n, w.window[1])
    with tdq.build_index(w.entries) as idx:
        with tdq.Plan(idx, n, result_capacity=16) as g, tdq.Plan(idx, n, use_graph=False) as nog:
            c1 = g.search(q, d, t0, t1)
            c2 = nog.search(q, d, t0, t1)
            assert c1 == c2 > 16
            _same(g.results(), nog.results())
            # replay the captured graph a few times: same answer
            for _ in range(3):
                assert g.search(q, d, t0, t1) == c1
            rg = g.results()
            _same(rg, nog.results())
        ref = tdq.search(idx, q, 15.0, *w.window)
    _same(rg, ref)


def test_plan_rejects_oversized_batches(tdq):
    rng = np.random.default_rng(5)
    ent = workloads.random_segments(rng, 100)
    q = workloads.random_segments(rng, 50)
    with tdq.build_index(ent) as idx, tdq.Plan(idx, 20) as plan:
        with pytest.raises(tdq.TdqError) as ei:
            plan.search(q, np.ones(50), np.zeros(50), np.full(50, 10.0))
        assert ei.value.status == tdq.TDQ_ERR_INVALID
        bad = q.take(np.arange(10))
        with pytest.raises(tdq.TdqError):
            plan.search(bad, np.full(10, -1.0), np.zeros(10), np.full(10, 10.0))
        assert plan.search(bad, np.ones(10), np.zeros(10), np.full(10, 10.0)) >= 0


def test_autotune_picks_measured_candidates(tdq):
    w = workloads.batching_walks(n_traj=800, n_queries=60, box=200.0)
    q = w.queries
    tun = tdq.autotune(w.entries, q, w.q_d, w.q_t0, w.q_t1, mode=tdq.MODE_FP32_FILTER, bin_counts=[500, 5000],
                       entry_chunks=[256, 512], batch_sizes=[1024, 2048], repeats=2)
    assert tun["bin_count"] in (500, 5000)
    assert tun["entry_chunk"] in (256, 512)
    assert tun["batch_query_segments"] in (1024, 2048, len(q))
    assert tun["ms_per_query_segment"] > 0
    # a plan with the tuned parameters returns the same results as an untuned one
    with tdq.build_index(w.entries, bin_count=tun["bin_count"]) as idx:
        b = int(tun["batch_query_segments"])
        with tdq.Plan(idx, b, mode=tdq.MODE_FP32_FILTER, entry_chunk=tun["entry_chunk"],
                      result_capacity=tun["result_capacity"]) as plan:
            parts = []
            for a in range(0, len(q), b):
                sl = np.arange(a, min(a + b, len(q)))
                plan.search(q.take(sl), w.q_d[sl], w.q_t0[sl], w.q_t1[sl])
                parts.append(plan.results())
        buf = tdq.DeviceResultBuffer(1 << 18)
        cnt = tdq.search_device_batched(idx, tdq.DeviceSegments(q), torch.from_numpy(w.q_d).cuda(),
                                        torch.from_numpy(w.q_t0).cuda(), torch.from_numpy(w.q_t1).cuda(), buf)
        ref = buf.to_host(cnt)
    merged = tdq.Results(*[np.concatenate([getattr(r, f) for r in parts])
                           for f in ("query_seg_id", "entry_seg_id", "t_enter", "t_exit")])
    _same(merged, ref)


def test_plan_results_into_caller_arrays(tdq):
    # results copied into caller-provided (pinned) host arrays equal the
    # freshly allocated copy; too small or mistyped arrays are refused
    w = workloads.tiny_random_walk()
    q = w.queries
    n = len(q)
    d = np.full(n, w.d_values[0])
    t0 = np.full(n, w.window[0])
    t1 = np.full(n, w.window[1])
    with tdq.build_index(w.entries) as idx, tdq.Plan(idx, n, mode=tdq.MODE_FP32_FILTER) as plan:
        c = plan.search(q, d, t0, t1)
        fresh = plan.results()
        cap = c + 5
        outs = tuple(torch.empty(cap, dtype=dt, pin_memory=True).numpy()
                     for dt in (torch.int64, torch.int64, torch.float64, torch.float64))
        got = plan.results(out=outs)
        assert len(got) == c > 0
        for f in ("query_seg_id", "entry_seg_id", "t_enter", "t_exit"):
            assert np.array_equal(getattr(got, f), getattr(fresh, f))
        with pytest.raises(ValueError):
            plan.results(out=tuple(a[: c - 1] for a in outs))
        with pytest.raises(ValueError):
            plan.results(out=(outs[2], outs[1], outs[2], outs[3]))
        # every overlapping pair a hit: 396,000 results, more than the
        # one-kernel copy's threads (grid-stride); then arrays of which one
        # is pageable (the copy-engine path)
        c = plan.search(q, np.full(n, 1e6), t0, t1)
        assert c == 20 * 99 * 200 == plan.stats()["overlap_pairs"]
        fresh = plan.results()
        big = tuple(torch.empty(c, dtype=dt, pin_memory=True).numpy()
                    for dt in (torch.int64, torch.int64, torch.float64, torch.float64))
        mixed = (big[0], big[1], np.empty(c, np.float64), big[3])
        for out in (big, mixed):
            got = plan.results(out=out)
            for f in ("query_seg_id", "entry_seg_id", "t_enter", "t_exit"):
                assert np.array_equal(getattr(got, f), getattr(fresh, f))


def _sorted(r):
    o = np.lexsort((r.entry_seg_id, r.query_seg_id))
    return r.query_seg_id[o], r.entry_seg_id[o], r.t_enter[o], r.t_exit[o]


def test_plan_with_host_results(tdq):
    # a plan whose result buffer is page-locked host memory: the kernels
    # write the results there, results(view=True) reads them in place (no
    # copy); the same items as a plan with a device buffer, in both modes,
    # also after the buffer overflowed and was regrown (every overlapping
    # pair a hit, 396,000 results); a device plan refuses view=True
    w = workloads.tiny_random_walk()
    q = w.queries
    n = len(q)
    t0 = np.full(n, w.window[0])
    t1 = np.full(n, w.window[1])
    with tdq.build_index(w.entries) as idx:
        for mode in (tdq.MODE_FP64, tdq.MODE_FP32_FILTER):
            with tdq.Plan(idx, n, mode=mode) as dev, tdq.Plan(idx, n, mode=mode, host_results=True) as host:
                for d in (w.d_values[0], 1e6):
                    dd = np.full(n, d)
                    c_dev = dev.search(q, dd, t0, t1)
                    c_host = host.search(q, dd, t0, t1)
                    assert c_dev == c_host > 0
                    ref = _sorted(dev.results())
                    got = host.results(view=True)
                    assert len(got) == c_host
                    for a, b in zip(ref, _sorted(got)):
                        assert np.array_equal(a, b)
                    for a, b in zip(ref, _sorted(host.results())):  # the copying path too
                        assert np.array_equal(a, b)
                assert c_host == 20 * 99 * 200
                with pytest.raises(ValueError):
                    dev.results(view=True)
                # the bench's end-to-end path: page-locked query arrays read
                # in place by the kernels, results read in place on the host
                def pinned(a):
                    p = torch.empty(len(a), dtype=torch.from_numpy(np.asarray(a)).dtype, pin_memory=True).numpy()
                    p[:] = a
                    return p

                qp = tdq.HostSegments(workloads.Segments(*[pinned(q[c]) for c in workloads.COLUMNS],
                                                         pinned(q.seg_id), pinned(q.traj_id)))
                dd = pinned(np.full(n, w.d_values[0]))
                c_dev = dev.search(q, np.full(n, w.d_values[0]), t0, t1)
                c_host = host.search(qp, dd, pinned(t0), pinned(t1))
                assert c_dev == c_host > 0
                for a, b in zip(_sorted(dev.results()), _sorted(host.results(view=True))):
                    assert np.array_equal(a, b)


def test_batching_workload_full_size_sampled(tdq):
    """The batching workload at full size (20,000 walks x 300 points = 5.98 M
    entries; 5,000 query trajectories with their own d and window, 449 k
    query segments) through one filter-mode plan with the batch size and
    entry chunk the autotuner picks for the benchmark; a seeded sample of 8
    query trajectories is checked pair by pair against the oracle."""
    w = workloads.batching_walks()
    q = w.queries
    n = len(q)
    batch = 42522
    with tdq.build_index(tdq.DeviceSegments(w.entries), bin_count=10000) as idx:
        qdev = tdq.DeviceSegments(q)
        dd, t0, t1 = (torch.from_numpy(a).cuda() for a in (w.q_d, w.q_t0, w.q_t1))
        got = []
        with tdq.Plan(idx, batch, mode=tdq.MODE_FP32_FILTER, entry_chunk=256) as plan:
            for a in range(0, n, batch):
                e = min(a + batch, n)
                sub = tdq.DeviceSegments(tensors=([c[a:e] for c in qdev.cols], qdev.seg_id[a:e], qdev.traj_id[a:e]))
                plan.search(sub, dd[a:e], t0[a:e], t1[a:e])
                got.append(plan.results())
    merged = tdq.Results(*[np.concatenate([getattr(r, f) for r in got])
                           for f in ("query_seg_id", "entry_seg_id", "t_enter", "t_exit")])
    # half of the sample among trajectories with results (pairs are rare:
    # ~0.007 per query segment), half at random; the oracle checks both ways
    rng = np.random.default_rng(11)
    seg_traj = dict(zip(q.seg_id.tolist(), q.traj_id.tolist()))
    with_hits = np.unique([seg_traj[s] for s in np.unique(merged.query_seg_id).tolist()])
    keep = np.unique(np.concatenate([rng.choice(with_hits, size=min(6, len(with_hits)), replace=False),
                                     rng.choice(np.unique(q.traj_id), size=6, replace=False)]))
    sel = np.nonzero(np.isin(q.traj_id, keep))[0]
    qs = q.take(sel)
    qd, q0, q1 = w.q_d[sel], w.q_t0[sel], w.q_t1[sel]
    mine = np.isin(merged.query_seg_id, qs.seg_id)
    gi = {"qi": _positions(merged.query_seg_id[mine], qs.seg_id),
          "ei": _positions(merged.entry_seg_id[mine], w.entries.seg_id),
          "t_enter": merged.t_enter[mine], "t_exit": merged.t_exit[mine]}
    ora = _oracle_per_trajectory(w, qs, qd, q0, q1)
    dmin = lambda ei, qi: oracle.pair_dmin(w.entries, ei, qs, qi, q0[qi], q1[qi])  # noqa: E731
    cmp = compare_results(gi, ora, w.entries, qs, None, dmin_fn=dmin, d_per_query=qd, win_per_query=(q0, q1))
    assert cmp["matched"] == len(ora["qi"]) > 0


def test_plan_reads_pinned_host_inputs_in_place(tdq):
    # page-locked host arrays are read in place by the replayed graph; the
    # results equal those of pageable host inputs (staged) and device inputs
    w = workloads.batching_walks(n_traj=300, n_queries=30, box=40.0)
    q = w.queries
    n = len(q)

    def pinned(a):
        p = torch.empty(len(a), dtype=torch.from_numpy(np.asarray(a)).dtype, pin_memory=True).numpy()
        p[:] = a
        return p

    qp = workloads.Segments(*[pinned(q[c]) for c in workloads.COLUMNS], pinned(q.seg_id), pinned(q.traj_id))
    with tdq.build_index(w.entries) as idx, tdq.Plan(idx, n, mode=tdq.MODE_FP32_FILTER) as plan:
        plan.search(q, w.q_d, w.q_t0, w.q_t1)
        staged = plan.results()
        plan.search(qp, pinned(w.q_d), pinned(w.q_t0), pinned(w.q_t1))
        in_place = plan.results()
        plan.search(tdq.DeviceSegments(q), torch.from_numpy(w.q_d).cuda(), torch.from_numpy(w.q_t0).cuda(),
                    torch.from_numpy(w.q_t1).cuda())
        device = plan.results()
    assert len(staged) > 0
    _same(in_place, staged)
    _same(device, staged)
