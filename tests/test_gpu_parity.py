"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Pair sets must be identical except for ties (pairs whose distance of closest
approach is within 1e-9*d of d); matched interval endpoints agree to 1e-9
relative (or, where a root is ill-conditioned, the reported time is still at
distance d within the same band)."""
import numpy as np
import pytest

from oracle import oracle
from paper_1405_7461_gb300 import workloads
from tests._util import GALAXY_ILL_CONDITIONED_MAX, compare_results, read_golden

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


def gpu_as_index(res, entries, queries):
    return {"qi": _positions(res.query_seg_id, queries.seg_id), "ei": _positions(res.entry_seg_id, entries.seg_id),
            "t_enter": res.t_enter, "t_exit": res.t_exit}


def oracle_as_dict(r):
    return {"qi": r.query_index, "ei": r.entry_index, "t_enter": r.t_enter, "t_exit": r.t_exit}


def check(tdq, entries, queries, d, t0=-np.inf, t1=np.inf, bin_count=0, brute=False, idx=None, max_ill=0, **params):
    own = idx is None
    if own:
        idx = tdq.build_index(entries, bin_count=bin_count)
    try:
        res = tdq.search(idx, queries, d, t0, t1, **params)
        stats = tdq.get_stats(idx)
    finally:
        if own:
            idx.free()
    ref = (oracle.search_bruteforce if brute else oracle.search_sweep)(entries, queries, d, t0, t1)
    cmp = compare_results(gpu_as_index(res, entries, queries), oracle_as_dict(ref), entries, queries, d, t0, t1,
                          dmin_fn=lambda ei, qi: oracle.pair_dmin(entries, ei, queries, qi, t0, t1),
                          max_ill_conditioned=max_ill)
    # the temporal-overlap count is exact integer work: identical
    assert stats["overlap_pairs"] == ref.overlap_pairs
    assert stats["interactions"] >= stats["overlap_pairs"] >= stats["results"] == len(res)
    return res, ref, stats, cmp


# --------------------------------------------------------------------------
# Index (Sec. 4, Fig. 1)
# --------------------------------------------------------------------------

def test_fig1_bin_table_on_gpu(tdq):
    g = read_golden("fig1_bins.txt")
    s = np.array(g["segments"])
    n = len(s)
    rng = np.random.default_rng(1)
    p0 = rng.uniform(0, 1, (n, 3))
    p1 = rng.uniform(0, 1, (n, 3))
    # present the segments in a shuffled order: the index must sort them
    perm = rng.permutation(n)
    seg = workloads.Segments(p0[perm, 0], p0[perm, 1], p0[perm, 2], s[perm, 1], p1[perm, 0], p1[perm, 1],
                             p1[perm, 2], s[perm, 2], s[perm, 0].astype(np.int64), np.zeros(n, np.int64))
    with tdq.build_index(seg, bin_count=4) as idx:
        bt = tdq.index_bins(idx, with_order=True)
    assert bt["width"] == 3.0 and bt["t_min"] == 0.0
    assert np.array_equal(seg.seg_id[bt["order"]], s[:, 0].astype(np.int64))
    for j, bstart, bend, bfirst, blast in g["bins"]:
        j = int(j)
        assert (bt["start"][j], bt["end"][j], bt["first"][j], bt["last"][j]) == (bstart, bend, int(bfirst),
                                                                                 int(blast))


def test_bin_table_matches_oracle_on_random_data(tdq):
    rng = np.random.default_rng(2)
    seg = workloads.random_segments(rng, 5000, t_span=50.0, max_dur=4.0)
    for m in (1, 7, 100, 4096):
        with tdq.build_index(seg, bin_count=m) as idx:
            bt = tdq.index_bins(idx, with_order=True)
        ref = oracle.bin_table(seg.ts, seg.te, m)
        assert np.array_equal(bt["order"], ref["order"])
        assert bt["width"] == ref["width"]
        assert np.array_equal(bt["first"], ref["first"])
        assert np.array_equal(bt["last"], ref["last"])
        ne = ref["first"] >= 0
        assert np.array_equal(bt["start"][ne], ref["start"][ne])
        assert np.array_equal(bt["end"][ne], ref["end"][ne])


# --------------------------------------------------------------------------
# Parity on the workloads
# --------------------------------------------------------------------------

def test_tiny_random_walk_parity(tdq):
    w = workloads.tiny_random_walk()
    res, ref, stats, cmp = check(tdq, w.entries, w.queries, 5.0, *w.window, brute=True)
    assert cmp["matched"] == len(ref.query_index) > len(w.queries)
    assert stats["overlap_pairs"] == 20 * 99 * 200


@pytest.mark.parametrize("seed,n,nq,chunk", [(3, 1, 1, 0), (4, 31, 33, 256), (5, 257, 65, 512), (6, 1000, 100, 2048),
                                              (7, 5000, 97, 1024), (8, 3000, 300, 256)])
def test_random_sets_ragged(tdq, seed, n, nq, chunk):
    rng = np.random.default_rng(seed)
    ent = workloads.random_segments(rng, n, box=8.0, t_span=20.0, max_dur=3.0)
    qry = workloads.random_segments(rng, nq, box=8.0, t_span=20.0, max_dur=3.0)
    qry.seg_id += 10 ** 9
    for d, win in ((1.5, (-np.inf, np.inf)), (0.7, (3.25, 14.5)), (4.0, (0.0, 5.0))):
        check(tdq, ent, qry, d, *win, bin_count=int(rng.integers(1, 300)), brute=True, entry_chunk=chunk)


@pytest.mark.parametrize("nq", [262_144, 262_145])
def test_query_sort_paths_at_the_small_path_limit(tdq, nq):
    # The query sort's small path (at most 256 tiles of 1024 keys; its digit
    # counts come from query_prep and the first scatter, no histogram kernel)
    # ends at 262,144 query segments; one more takes the general path
    # (histogram and scan kernels).  Both against the oracle, in both modes,
    # directly and through a batched plan (whose graph sorts the padded size
    # class: 262,144 and 524,288), with a window that empties some segments.
    rng = np.random.default_rng(nq)
    ent = workloads.random_segments(rng, 4000, box=30.0, t_span=2000.0, max_dur=3.0)
    qry = workloads.random_segments(rng, nq, box=30.0, t_span=2000.0, max_dur=3.0)
    qry.seg_id += 10 ** 9
    t0, t1 = 10.0, 1990.0
    with tdq.build_index(ent, bin_count=500) as idx:
        for mode in (tdq.MODE_FP64, tdq.MODE_FP32_FILTER):
            res, ref, stats, cmp = check(tdq, ent, qry, 2.0, t0, t1, idx=idx, mode=mode)
            assert cmp["matched"] > 1000
            with tdq.Plan(idx, nq, mode=mode, result_capacity=1 << 20) as plan:
                cnt = plan.search(qry, np.full(nq, 2.0), np.full(nq, t0), np.full(nq, t1))
                assert cnt == len(res)
                assert plan.stats()["overlap_pairs"] == ref.overlap_pairs
                for a, b in zip(_sorted_arrays(res), _sorted_arrays(plan.results())):
                    assert np.array_equal(a, b)


def test_scale_random_walk_reduced(tdq):
    w = workloads.scale_random_walk(n_traj=1500, n_queries=25)
    with tdq.build_index(w.entries) as idx:
        for d in w.d_values:
            check(tdq, w.entries, w.queries, d, *w.window, idx=idx)


def test_scale_random_walk_full_size(tdq):
    """The benchmark workload at full size (10,000 walks, 100 queries) in the
    launch configuration the benchmark times, every d, every pair."""
    w = workloads.scale_random_walk()
    with tdq.build_index(w.entries) as idx:
        for d in w.d_values:
            res, ref, stats, cmp = check(tdq, w.entries, w.queries, d, *w.window, idx=idx)
            assert stats["overlap_pairs"] > 1e8


def test_galaxy_disk_near_tangent(tdq):
    w = workloads.galaxy_disk(n_stars=3000, n_queries=30)
    with tdq.build_index(w.entries) as idx:
        for d in w.d_values:
            check(tdq, w.entries, w.queries, d, *w.window, idx=idx, max_ill=GALAXY_ILL_CONDITIONED_MAX)


def test_galaxy_disk_full_size_sampled(tdq):
    """Full-size galaxy database (9.95 M segments); a seeded sample of 20
    query trajectories is checked pair by pair against the oracle."""
    w = workloads.galaxy_disk()
    rng = np.random.default_rng(5)
    keep = rng.choice(np.unique(w.queries.traj_id), size=20, replace=False)
    q = w.queries.take(np.nonzero(np.isin(w.queries.traj_id, keep))[0])
    with tdq.build_index(w.entries) as idx:
        for d in w.d_values:
            check(tdq, w.entries, q, d, *w.window, idx=idx, max_ill=GALAXY_ILL_CONDITIONED_MAX)


def test_batched_per_query_threshold_and_window(tdq):
    w = workloads.batching_walks(n_traj=400, n_queries=60, box=40.0)
    q = w.queries
    qdev = tdq.DeviceSegments(q)
    dd = torch.from_numpy(w.q_d).cuda()
    t0 = torch.from_numpy(w.q_t0).cuda()
    t1 = torch.from_numpy(w.q_t1).cuda()
    buf = tdq.DeviceResultBuffer(1 << 18)
    with tdq.build_index(w.entries, bin_count=3000) as idx:
        cnt = tdq.search_device_batched(idx, qdev, dd, t0, t1, buf)
        res = buf.to_host(cnt)
    got = gpu_as_index(res, w.entries, q)
    # oracle: one search per query trajectory with its own d and window
    parts = {k: [] for k in ("qi", "ei", "t_enter", "t_exit")}
    for tj in np.unique(q.traj_id):
        sel = np.nonzero(q.traj_id == tj)[0]
        r = oracle.search_sweep(w.entries, q.take(sel), w.q_d[sel[0]], w.q_t0[sel[0]], w.q_t1[sel[0]])
        parts["qi"].append(sel[r.query_index])
        parts["ei"].append(r.entry_index)
        parts["t_enter"].append(r.t_enter)
        parts["t_exit"].append(r.t_exit)
    ref = {k: np.concatenate(v) for k, v in parts.items()}
    dmin = lambda ei, qi: oracle.pair_dmin(w.entries, ei, q, qi, w.q_t0[qi], w.q_t1[qi])  # noqa: E731
    cmp = compare_results(got, ref, w.entries, q, None, dmin_fn=dmin, d_per_query=w.q_d,
                          win_per_query=(w.q_t0, w.q_t1))
    assert cmp["matched"] > 1000


# --------------------------------------------------------------------------
# Edge cases and the boundary's error behaviour
# --------------------------------------------------------------------------

def _segs(rows, ids=None):
    a = np.array(rows, np.float64).reshape(-1, 8)
    return workloads.Segments.from_columns([a[:, k] for k in range(8)], seg_id=ids)


def test_host_results_stay_valid_while_held(tdq):
    # library-owned host results live in recycled page-locked blocks: a result
    # set still held is never handed out again, and later searches (reusing
    # released blocks of the same size class) leave it intact
    import gc
    w = workloads.tiny_random_walk()
    with tdq.build_index(w.entries) as idx:
        a = tdq.search(idx, w.queries, 5.0, *w.window)
        keep_a = [x.copy() for x in _sorted_arrays(a)]
        b = tdq.search(idx, w.queries, 5.0, *w.window)
        assert a.query_seg_id.ctypes.data != b.query_seg_id.ctypes.data
        keep_b = [x.copy() for x in _sorted_arrays(b)]
        for x, y in zip(keep_a, keep_b):
            assert np.array_equal(x, y)
        del a
        gc.collect()
        for _ in range(3):  # reuse a's block with other contents
            c = tdq.search(idx, w.queries, 2.5, *w.window)
            assert 0 < len(c) < len(b)
        for x, y in zip(keep_b, _sorted_arrays(b)):
            assert np.array_equal(x, y)


def test_empty_inputs(tdq):
    rng = np.random.default_rng(9)
    ent = workloads.random_segments(rng, 100)
    empty = workloads.random_segments(rng, 0)
    with tdq.build_index(ent) as idx:
        assert len(tdq.search(idx, empty, 1.0)) == 0
    with tdq.build_index(empty) as idx:
        assert tdq.index_size(idx) == 0
        assert len(tdq.search(idx, ent, 1.0)) == 0


def test_window_outside_data_and_touching_segments(tdq):
    rng = np.random.default_rng(10)
    ent = workloads.random_segments(rng, 500, t_span=10.0)
    with tdq.build_index(ent) as idx:
        assert len(tdq.search(idx, ent, 100.0, 50.0, 60.0)) == 0
        assert len(tdq.search(idx, ent, 100.0, 3.0, 3.0)) == 0  # zero-length window
    # a walk's own consecutive segments touch only at instants
    e = _segs([[0, 0, 0, 0, 1, 0, 0, 1], [1, 0, 0, 1, 2, 0, 0, 2]])
    q = _segs([[1, 0, 0, 1, 2, 0, 0, 2]], ids=[77])
    with tdq.build_index(e) as idx:
        r = tdq.search(idx, q, 5.0)
    assert r.entry_seg_id.tolist() == [1] and (r.t_enter[0], r.t_exit[0]) == (1.0, 2.0)


def test_zero_threshold_self_match_and_duplicates(tdq):
    w = workloads.tiny_random_walk(n_traj=30, n_points=20, n_queries=3)
    e = workloads.Segments.concat([w.entries, w.entries.take(np.arange(len(w.entries)))])
    e.seg_id = np.arange(len(e), dtype=np.int64)
    res, ref, stats, cmp = check(tdq, e, w.queries, 0.0, brute=True)
    # each query segment matches itself and its duplicate, over its whole extent
    assert len(res) >= 2 * len(w.queries)


def test_invalid_inputs_are_rejected(tdq):
    rng = np.random.default_rng(12)
    ent = workloads.random_segments(rng, 50)
    bad = workloads.random_segments(rng, 50)
    bad.te[7] = bad.ts[7]
    with pytest.raises(tdq.TdqError) as ei:
        tdq.build_index(bad)
    assert ei.value.status == tdq.TDQ_ERR_INVALID
    nanq = workloads.random_segments(rng, 40)
    nanq.xs[3] = np.nan
    with tdq.build_index(ent) as idx:
        for args in ((nanq, 1.0), (ent, -1.0), (ent, np.nan), (ent, np.inf)):
            with pytest.raises(tdq.TdqError) as ei:
                tdq.search(idx, *args)
            assert ei.value.status == tdq.TDQ_ERR_INVALID
        with pytest.raises(tdq.TdqError):
            tdq.search(idx, ent, 1.0, 5.0, 2.0)
        # the index is still usable after rejected calls
        assert len(tdq.search(idx, ent, 1.0)) >= len(ent)


def test_result_overflow_and_retry(tdq):
    """A cluster where every pair is in range: the device call reports the
    needed size, and the host call grows its buffer and re-runs (Sec. 5)."""
    rng = np.random.default_rng(13)
    n, nq = 3000, 40
    ent = workloads.random_segments(rng, n, box=0.1, t_span=0.5, max_dur=20.0, max_speed=0.01)
    qry = workloads.random_segments(rng, nq, box=0.1, t_span=0.5, max_dur=20.0, max_speed=0.01)
    qry.seg_id += 10 ** 6
    need = n * nq
    with tdq.build_index(ent) as idx:
        qd = tdq.DeviceSegments(qry)
        small = tdq.DeviceResultBuffer(1)
        cnt = tdq.search_device(idx, qd, 5.0, -np.inf, np.inf, small, allow_overflow=True)
        assert cnt == need
        with pytest.raises(tdq.TdqError) as ei:
            tdq.search_device(idx, qd, 5.0, -np.inf, np.inf, small)
        assert ei.value.status == tdq.TDQ_ERR_OVERFLOW
        res = tdq.search(idx, qry, 5.0)  # internal buffer starts at 65,536 < 120,000 items
        assert len(res) == need
        big = tdq.DeviceResultBuffer(need)
        cnt = tdq.search_device(idx, qd, 5.0, -np.inf, np.inf, big)
        r2 = big.to_host(cnt)
    k1 = np.sort(res.query_seg_id * (1 << 32) + res.entry_seg_id)
    k2 = np.sort(r2.query_seg_id * (1 << 32) + r2.entry_seg_id)
    assert np.array_equal(k1, k2)


def test_host_and_device_calls_agree(tdq):
    w = workloads.scale_random_walk(n_traj=800, n_queries=10)
    with tdq.build_index(tdq.DeviceSegments(w.entries)) as idx:
        a = tdq.search(idx, w.queries, 15.0, *w.window)
        buf = tdq.DeviceResultBuffer(len(a) + 10)
        cnt = tdq.search_device(idx, tdq.DeviceSegments(w.queries), 15.0, *w.window, buf)
        b = buf.to_host(cnt)
    oa = np.lexsort((a.entry_seg_id, a.query_seg_id))
    ob = np.lexsort((b.entry_seg_id, b.query_seg_id))
    for f in ("query_seg_id", "entry_seg_id", "t_enter", "t_exit"):
        assert np.array_equal(getattr(a, f)[oa], getattr(b, f)[ob])


# --------------------------------------------------------------------------
# FP32 conservative pre-test + FP64 refinement (filter mode)
# --------------------------------------------------------------------------

def _sorted_arrays(r):
    o = np.lexsort((r.entry_seg_id, r.query_seg_id))
    return r.query_seg_id[o], r.entry_seg_id[o], r.t_enter[o], r.t_exit[o]


FILTER_MODES = ["fp32filter", "tcfilter"]


def _mode(tdq, name):
    return {"fp64": tdq.MODE_FP64, "fp32filter": tdq.MODE_FP32_FILTER, "tcfilter": tdq.MODE_TC_FILTER}[name]


def _filter_vs_fp64(tdq, idx, queries, d, window, mode="fp32filter"):
    r64 = tdq.search(idx, queries, d, *window, mode=tdq.MODE_FP64)
    s64 = tdq.get_stats(idx)
    r32 = tdq.search(idx, queries, d, *window, mode=_mode(tdq, mode))
    s32 = tdq.get_stats(idx)
    # the filter drops only pairs the FP64 test rejects, and survivors run the
    # same FP64 code: the results are bitwise identical
    for a, b in zip(_sorted_arrays(r64), _sorted_arrays(r32)):
        assert np.array_equal(a, b)
    assert s32["overlap_pairs"] == s64["overlap_pairs"] == s64["fp64_pairs"]
    assert s32["results"] <= s32["fp64_pairs"] <= s32["overlap_pairs"]
    return s64, s32


@pytest.mark.parametrize("mode", FILTER_MODES)
@pytest.mark.parametrize("name", ["tiny", "scale", "galaxy", "batching"])
def test_filter_mode_equals_plain_fp64(tdq, name, mode):
    if name == "tiny":
        w = workloads.tiny_random_walk()
    elif name == "scale":
        w = workloads.scale_random_walk(n_traj=2000, n_queries=20)
    elif name == "galaxy":
        w = workloads.galaxy_disk(n_stars=4000, n_queries=25)
    else:
        w = workloads.batching_walks(n_traj=500, n_queries=40, box=60.0)
        w.d_values = (0.5, 4.0, 10.0)
    with tdq.build_index(w.entries) as idx:
        for d in w.d_values:
            s64, s32 = _filter_vs_fp64(tdq, idx, w.queries, d, w.window, mode)
        # and against the oracle, through the filter path
        check(tdq, w.entries, w.queries, w.d_values[-1], *w.window, idx=idx, mode=_mode(tdq, mode),
              max_ill=GALAXY_ILL_CONDITIONED_MAX if name == "galaxy" else 0)


@pytest.mark.parametrize("mode", FILTER_MODES)
def test_filter_mode_full_size_scale_walk(tdq, mode):
    w = workloads.scale_random_walk()
    with tdq.build_index(w.entries) as idx:
        for d in w.d_values:
            s64, s32 = _filter_vs_fp64(tdq, idx, w.queries, d, w.window, mode)
            assert s32["fp64_pairs"] < 0.01 * s32["overlap_pairs"]


@pytest.mark.parametrize("mode", FILTER_MODES)
@pytest.mark.parametrize("offset", [0.0, 1e3, 1e5, 3e6])
def test_filter_is_conservative_at_the_threshold(tdq, offset, mode):
    """Pairs whose closest distance is d(1 - 1e-7) .. d(1 + 1e-7), far from
    the origin where FP32 rounding is coarse: the filter must keep every
    pair the FP64 test accepts (the two modes agree pair for pair)."""
    rng = np.random.default_rng(int(offset) + 17)
    n = 4000
    d = 0.75
    rel = rng.uniform(-1e-7, 1e-7, n)
    # query: a point moving along x through the origin region (plus offset)
    q = np.array([[offset - 5.0, offset, offset, 0.0, offset + 5.0, offset, offset, 10.0]])
    # entries: stationary points at distance d(1+rel) from the query's line,
    # each over a span that contains its closest-approach time
    u = rng.normal(size=(n, 2))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    x = offset + rng.uniform(-4.0, 4.0, n)
    y = offset + u[:, 0] * d * (1 + rel)
    z = offset + u[:, 1] * d * (1 + rel)
    t0 = rng.uniform(0.0, 1.0, n)  # spans hold the closest approach (t in [1, 9])
    t1 = rng.uniform(9.0, 10.0, n)
    ent = workloads.Segments.from_columns([x, y, z, t0, x, y, z, t1])
    qry = workloads.Segments.from_columns([q[:, k] for k in range(8)], seg_id=[10 ** 9])
    with tdq.build_index(ent) as idx:
        s64, s32 = _filter_vs_fp64(tdq, idx, qry, d, (-np.inf, np.inf), mode)
    assert s64["results"] > 0.3 * n


@pytest.mark.parametrize("mode", FILTER_MODES)
@pytest.mark.parametrize("offset", [0.0, 1e3, 1e5, 3e6])
def test_filter_keeps_touching_stationary_spheres(tdq, offset, mode):
    """Stationary query and entry points (zero-radius spheres) at distance
    d (1 + rel), rel in [-1e-7, 1e-7]: the sphere test is then as tight as the
    FP64 decision itself, so the pre-test's margin alone keeps the pairs the
    FP64 test accepts (the two modes agree pair for pair)."""
    rng = np.random.default_rng(int(offset) + 29)
    n = 3000
    d = 0.625
    rel = rng.uniform(-1e-7, 1e-7, n)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    c = offset + 7.0 + u * (d * (1 + rel))[:, None]
    # a spread of other stationary entries, so that the grid is not centred
    # on the query
    far = offset + rng.uniform(-40.0, 60.0, (n, 3))
    p = np.concatenate([c, far])
    t0 = np.zeros(2 * n)
    t1 = np.full(2 * n, 4.0)
    ent = workloads.Segments.from_columns([p[:, 0], p[:, 1], p[:, 2], t0, p[:, 0], p[:, 1], p[:, 2], t1])
    q = np.array([offset + 7.0, offset + 7.0, offset + 7.0, 1.0, offset + 7.0, offset + 7.0, offset + 7.0, 3.0])
    qry = workloads.Segments.from_columns([q[[k]] for k in range(8)], seg_id=[10 ** 9])
    with tdq.build_index(ent) as idx:
        s64, s32 = _filter_vs_fp64(tdq, idx, qry, d, (-np.inf, np.inf), mode)
    assert 0.3 * n < s64["results"] < 0.7 * n


@pytest.mark.parametrize("mode", FILTER_MODES)
def test_filter_survivor_list_overflow_is_regrown(tdq, mode):
    """A cluster where every pair survives the pre-test: 1.3 M survivors
    overflow the initial survivor list (2^20 pairs), which is grown and the
    search re-run; the results equal the plain FP64 mode's.  (64 query
    segments: a small search, whose FP32 pre-test refines the survivors in
    place instead -- up to 4,096 in a pass of 128 entries, which fill its
    warp's buffer in rounds.)"""
    rng = np.random.default_rng(21)
    ent = workloads.random_segments(rng, 20_000, box=0.2, t_span=0.5, max_dur=20.0, max_speed=0.01)
    qry = workloads.random_segments(rng, 64, box=0.2, t_span=0.5, max_dur=20.0, max_speed=0.01)
    qry.seg_id += 10 ** 7
    with tdq.build_index(ent) as idx:
        s64, s32 = _filter_vs_fp64(tdq, idx, qry, 3.0, (-np.inf, np.inf), mode)
    assert s32["results"] == 20_000 * 64


@pytest.mark.parametrize("bin_count", [1, 3, 64, 4096, 100_000])
def test_filter_overlap_count_across_bins_and_windows(tdq, bin_count):
    # the filter mode counts temporal-overlap pairs with searches confined to
    # the bin of each bound (t_start table and t_end table): the count must be
    # the oracle's for any bin width -- one bin, bins much wider and much
    # narrower than a segment -- and for windows inside, cutting, before and
    # after the data
    w = workloads.scale_random_walk(n_traj=300, n_queries=12)
    ts = np.concatenate([w.entries["ts"], w.entries["te"]])
    lo, hi = float(ts.min()), float(ts.max())
    mid = 0.5 * (lo + hi)
    windows = [(-np.inf, np.inf), (mid - 7.25, mid + 3.5), (lo - 50.0, lo + 0.5), (hi - 0.25, hi + 10.0),
               (lo - 20.0, lo - 10.0), (hi + 1.0, hi + 2.0)]
    with tdq.build_index(w.entries, bin_count=bin_count) as idx:
        for t0, t1 in windows:
            r64 = tdq.search(idx, w.queries, 5.0, t0, t1, mode=tdq.MODE_FP64)
            s64 = tdq.get_stats(idx)
            ref = oracle.search_sweep(w.entries, w.queries, 5.0, t0, t1)
            for mode in (tdq.MODE_FP32_FILTER, tdq.MODE_TC_FILTER):
                r32 = tdq.search(idx, w.queries, 5.0, t0, t1, mode=mode)
                s32 = tdq.get_stats(idx)
                assert s32["overlap_pairs"] == s64["overlap_pairs"] == ref.overlap_pairs
                for a, b in zip(_sorted_arrays(r64), _sorted_arrays(r32)):
                    assert np.array_equal(a, b)
                assert len(r32) == len(ref.query_index)


# --------------------------------------------------------------------------
# Self-join: query (ii) of Sec. 2.1 with the database as the query set
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,mode", [("tiny", "fp64"), ("tiny", "fp32filter"), ("tiny", "tcfilter"),
                                       ("galaxy", "fp32filter"), ("galaxy", "tcfilter"), ("galaxy", "fp64")])
def test_self_join_matches_oracle(tdq, name, mode):
    if name == "tiny":
        w = workloads.tiny_random_walk(n_traj=120, n_points=60)
        d, window = 6.0, (-np.inf, np.inf)
    else:
        w = workloads.galaxy_disk(n_stars=300, n_queries=1)
        d, window = 0.1, (20.0, 120.5)
    ent = w.entries
    # ids unrelated to positions, so that "each unordered pair once" is not
    # an artefact of the sort order
    ent.seg_id = ent.seg_id[np.random.default_rng(5).permutation(len(ent))]
    m = _mode(tdq, mode)
    with tdq.build_index(ent) as idx:
        res = tdq.self_join(idx, ent, d, *window, mode=m)
        stats = tdq.get_stats(idx)
    ref = oracle.self_join(ent, d, *window)
    assert stats["overlap_pairs"] == ref.overlap_pairs
    assert np.all(res.query_seg_id < res.entry_seg_id)
    cmp = compare_results(gpu_as_index(res, ent, ent), oracle_as_dict(ref), ent, ent, d, *window,
                          dmin_fn=lambda ei, qi: oracle.pair_dmin(ent, ei, ent, qi, *window),
                          max_ill_conditioned=GALAXY_ILL_CONDITIONED_MAX if name == "galaxy" else 0)
    assert cmp["matched"] == len(ref.query_index) > 0


def test_pair_filter_arguments_are_checked(tdq):
    w = workloads.tiny_random_walk(n_traj=20, n_points=10)
    ent = w.entries
    with tdq.build_index(ent) as idx:
        with pytest.raises(tdq.TdqError):  # unknown flag bit
            tdq.search(idx, ent, 1.0, flags=4)
        with pytest.raises(tdq.TdqError):  # a different segment set than the index's
            tdq.self_join(idx, ent.take(np.arange(len(ent) - 1)), 1.0)
        # the flags alone, on a host query set without trajectory ids
        q = ent.take(np.arange(50))
        s = tdq.HostSegments(q)
        st = s.struct()
        st.traj_id = None
        out = tdq.ctypes.POINTER(tdq.tdq_results)()
        prm = tdq._params(flags=tdq.FLAG_OTHER_TRAJECTORIES)
        rc = tdq.load().tdq_search(idx.handle, tdq.ctypes.byref(st), 1.0, -np.inf, np.inf, tdq.ctypes.byref(prm),
                                   None, tdq.ctypes.byref(out))
        assert rc == tdq.TDQ_ERR_INVALID
        # filters on an ordinary search: same as the self-join
        a = tdq.search(idx, ent, 3.0, flags=tdq.FLAG_OTHER_TRAJECTORIES | tdq.FLAG_UNORDERED_ONCE,
                       mode=tdq.MODE_FP32_FILTER)
        b = tdq.self_join(idx, ent, 3.0)
        for x, y in zip(_sorted_arrays(a), _sorted_arrays(b)):
            assert np.array_equal(x, y)


def test_pinned_host_queries_are_read_in_place(tdq):
    # tdq_search reads page-locked host query arrays in place (no staging
    # copy); the results equal those of the same queries in pageable memory
    torch = pytest.importorskip("torch")
    w = workloads.scale_random_walk(n_traj=600, n_queries=8)

    def pinned(a):
        p = torch.empty(len(a), dtype=torch.from_numpy(np.asarray(a)).dtype, pin_memory=True).numpy()
        p[:] = a
        return p

    qp = workloads.Segments(*[pinned(w.queries[c]) for c in workloads.COLUMNS], pinned(w.queries.seg_id),
                            pinned(w.queries.traj_id))
    with tdq.build_index(w.entries) as idx:
        for mode in (tdq.MODE_FP64, tdq.MODE_FP32_FILTER):
            a = tdq.search(idx, w.queries, 5.0, *w.window, mode=mode)
            b = tdq.search(idx, qp, 5.0, *w.window, mode=mode)
            assert len(a) > 0
            for x, y in zip(_sorted_arrays(a), _sorted_arrays(b)):
                assert np.array_equal(x, y)


def test_filter_with_magnitudes_beyond_two_to_the_sixty(tdq):
    # segments beyond 2^60 in magnitude get an infinite bounding radius (and
    # E or K = -inf): the pre-test never rejects them; mixed with ordinary
    # segments, the filter mode must still return exactly the plain FP64 set
    rng = np.random.default_rng(21)
    far = workloads.random_segments(rng, 3000, box=2e5, t_span=20.0, max_dur=3.0, max_speed=5e3)
    near = workloads.random_segments(rng, 3000, box=200.0, t_span=20.0, max_dur=3.0, max_speed=5.0)
    shift = 3e18  # > 2^60 = 1.15e18
    for c in ("xs", "xe"):
        setattr(far, c, getattr(far, c) + shift)
    ent = workloads.Segments.concat([far, near])
    ent.seg_id = np.arange(len(ent), dtype=np.int64)
    ent.traj_id = np.arange(len(ent), dtype=np.int64)
    q = ent.take(np.concatenate([np.arange(0, 3000, 60), np.arange(3000, 6000, 60)]))
    with tdq.build_index(ent) as idx:
        for d in (50.0, 3e4):
            r64 = tdq.search(idx, q, d, mode=tdq.MODE_FP64)
            for mode in (tdq.MODE_FP32_FILTER, tdq.MODE_TC_FILTER):
                r32 = tdq.search(idx, q, d, mode=mode)
                s32 = tdq.get_stats(idx)
                for a, b in zip(_sorted_arrays(r64), _sorted_arrays(r32)):
                    assert np.array_equal(a, b)
                assert len(r32) >= len(q)  # every query segment meets itself
                assert s32["fp64_pairs"] > 0
