"""The tensor-core pre-test (TDQ_MODE_TC_FILTER) at the edges of its integer
grid.  The pre-test may only drop pairs whose bounding spheres cannot meet;
everything else goes to the FP64 evaluation of Sec. 5 / Algorithm 1, so the
mode must return bitwise the plain FP64 mode's pairs and intervals.  These
cases push the grid: coordinates at its corners, radii near and beyond its
largest representable radius, queries outside the entries' box (clamped),
entries too long for the grid, a box of zero extent, and query counts that
leave the last supertile of 128 ragged."""
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


def _sorted(r):
    o = np.lexsort((r.entry_seg_id, r.query_seg_id))
    return r.query_seg_id[o], r.entry_seg_id[o], r.t_enter[o], r.t_exit[o]


def _same_as_fp64(tdq, idx, q, d, t0=-np.inf, t1=np.inf):
    r64 = tdq.search(idx, q, d, t0, t1, mode=tdq.MODE_FP64)
    s64 = tdq.get_stats(idx)
    rtc = tdq.search(idx, q, d, t0, t1, mode=tdq.MODE_TC_FILTER)
    stc = tdq.get_stats(idx)
    for a, b in zip(_sorted(r64), _sorted(rtc)):
        assert np.array_equal(a, b)
    assert stc["overlap_pairs"] == s64["overlap_pairs"]
    assert stc["results"] <= stc["fp64_pairs"] <= stc["filter_survivors"]
    return r64, s64, stc


def _segs(p0, p1, t0, t1, first_id=0):
    p0 = np.asarray(p0, np.float64)
    p1 = np.asarray(p1, np.float64)
    n = len(p0)
    return workloads.Segments.from_columns([p0[:, 0], p0[:, 1], p0[:, 2], np.broadcast_to(t0, n).copy(), p1[:, 0],
                                            p1[:, 1], p1[:, 2], np.broadcast_to(t1, n).copy()],
                                           seg_id=np.arange(first_id, first_id + n))


def test_grid_corners_and_largest_radii(tdq):
    # entries fill [0,100]^3 with the 8 corners among them (grid coordinates
    # +-1023); queries at corners and centre with d up to and beyond the
    # largest grid radius (1023 units = 50 at this extent)
    rng = np.random.default_rng(3)
    n = 4000
    p = rng.uniform(0.0, 100.0, (n, 3))
    corners = np.array([[x, y, z] for x in (0.0, 100.0) for y in (0.0, 100.0) for z in (0.0, 100.0)])
    p[:8] = corners
    step = rng.normal(0.0, 0.3, (n, 3))
    ent = _segs(p, p + step, 0.0, 10.0)
    qp = np.concatenate([corners, [[50.0, 50.0, 50.0]]])
    qry = _segs(qp, qp + 0.5, 2.0, 8.0, first_id=10 ** 6)
    with tdq.build_index(ent) as idx:
        for d in (0.5, 12.0, 47.0, 49.9, 60.0, 400.0):
            r64, s64, stc = _same_as_fp64(tdq, idx, qry, d)
            assert len(r64) >= 8  # every corner query meets its corner entry
            if d >= 60.0:  # radius beyond the grid: every overlapping pair survives
                assert stc["filter_survivors"] == s64["overlap_pairs"]


def test_queries_outside_the_entries_box_are_clamped(tdq):
    # entries in [0,10]^3, queries around (100,100,100) and (-80, 5, 5): their
    # grid centres are clamped to the box, which only shortens distances
    rng = np.random.default_rng(4)
    p = rng.uniform(0.0, 10.0, (3000, 3))
    ent = _segs(p, p + rng.normal(0.0, 0.1, p.shape), 0.0, 5.0)
    qp = np.concatenate([100.0 + rng.uniform(-3, 3, (40, 3)), np.array([-80.0, 5.0, 5.0]) + rng.uniform(-3, 3, (40, 3))])
    qry = _segs(qp, qp + rng.normal(0.0, 0.2, qp.shape), 1.0, 4.0, first_id=10 ** 6)
    with tdq.build_index(ent) as idx:
        for d in (85.0, 151.0, 160.0):
            r64, _, _ = _same_as_fp64(tdq, idx, qry, d)
        assert len(r64) > 0


def test_entries_too_long_for_the_grid_always_survive(tdq):
    # a few segments thousands of units long among short ones: their grid
    # radius exceeds the largest, so they pass the pre-test against every query
    rng = np.random.default_rng(5)
    p = rng.uniform(0.0, 50.0, (2000, 3))
    e = p + rng.normal(0.0, 0.5, p.shape)
    e[:5] = p[:5] + np.array([4000.0, -3000.0, 2500.0])
    ent = _segs(p, e, 0.0, 8.0)
    qry = ent.take(np.arange(0, 2000, 37))
    qry.seg_id = qry.seg_id + 10 ** 6
    with tdq.build_index(ent) as idx:
        for d in (0.7, 3.0):
            _same_as_fp64(tdq, idx, qry, d)


def test_entries_at_one_point(tdq):
    # zero extent: every entry centre maps to the grid origin
    n = 500
    p = np.full((n, 3), 12.5)
    ent = _segs(p, p, np.arange(n) * 0.01, np.arange(n) * 0.01 + 3.0)
    qp = np.array([[12.5, 12.5, 12.5], [13.0, 12.5, 12.5], [20.0, 0.0, 0.0]])
    qry = _segs(qp, qp, 0.5, 4.0, first_id=10 ** 6)
    with tdq.build_index(ent) as idx:
        for d in (0.0, 0.4, 0.5, 30.0):
            _same_as_fp64(tdq, idx, qry, d)


@pytest.mark.parametrize("nq", [1, 31, 127, 128, 129, 300, 1000])
def test_ragged_supertiles_against_the_oracle(tdq, nq):
    rng = np.random.default_rng(100 + nq)
    ent = workloads.random_segments(rng, 5000, box=30.0, t_span=20.0, max_dur=3.0)
    qry = workloads.random_segments(rng, nq, box=30.0, t_span=20.0, max_dur=3.0)
    qry.seg_id = qry.seg_id + 10 ** 6
    d = 2.5
    with tdq.build_index(ent) as idx:
        _same_as_fp64(tdq, idx, qry, d)
        res = tdq.search(idx, qry, d, mode=tdq.MODE_TC_FILTER)
    ref = oracle.search_sweep(ent, qry, d)
    qo = np.argsort(qry.seg_id)
    got = {"qi": qo[np.searchsorted(qry.seg_id[qo], res.query_seg_id)], "ei": res.entry_seg_id.copy(),
           "t_enter": res.t_enter, "t_exit": res.t_exit}
    cmp = compare_results(got, {"qi": ref.query_index, "ei": ref.entry_index, "t_enter": ref.t_enter,
                                "t_exit": ref.t_exit}, ent, qry, d,
                          dmin_fn=lambda ei, qi: oracle.pair_dmin(ent, ei, qry, qi))
    assert cmp["matched"] == len(ref.query_index)


def test_selectivity_on_the_scale_walk(tdq):
    # the grid's rounding widens the spheres by at most (sqrt(3) + 2) grid
    # units (about 1 unit of length here): the tensor-core pre-test passes at
    # most a few times the FP32 pre-test's survivors, not every candidate
    w = workloads.scale_random_walk(n_traj=3000, n_queries=30)
    with tdq.build_index(w.entries) as idx:
        for d in w.d_values:
            tdq.search(idx, w.queries, d, *w.window, mode=tdq.MODE_FP32_FILTER)
            s32 = tdq.get_stats(idx)
            _, _, stc = _same_as_fp64(tdq, idx, w.queries, d, *w.window)
            assert stc["filter_survivors"] <= 4 * s32["filter_survivors"] + 1000
            assert stc["filter_survivors"] < 0.01 * stc["interactions"]
