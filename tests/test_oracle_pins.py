"""Pins for the CPU FP64 oracle: closed forms, invariants, dense time sampling,
brute force against the sweep, and the paper's index example (Fig. 1).

Each check is derived from the mathematics of moving points or from numbers
printed in the paper, never from the oracle's own formula."""
import math

import numpy as np
import pytest

from oracle import oracle
from paper_1405_7461_gb300 import workloads
from tests._util import dist_at, read_golden


def seg(p0, t0, p1, t1):
    return np.array([p0[0], p0[1], p0[2], t0, p1[0], p1[1], p1[2], t1], np.float64)


def moving(p_at_0, v, t0, t1):
    """Segment of a point with position p_at_0 + v t, over [t0, t1]."""
    p_at_0 = np.asarray(p_at_0, float)
    v = np.asarray(v, float)
    return seg(p_at_0 + v * t0, t0, p_at_0 + v * t1, t1)


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("frac,hit", [(0.0, True), (0.5, True), (1.0 - 1e-6, True), (1.0 + 1e-6, False),
                                      (2.0, False)])
def test_stationary_point_query(frac, hit):
    """Sec. 2.1 query (i): a non-moving point over an interval.  A stationary
    entry at distance r is in range over the whole common span iff r <= d."""
    d = 3.0
    q = seg((1.0, 2.0, 3.0), 2.0, (1.0, 2.0, 3.0), 8.0)
    direction = np.array([2.0, -1.0, 2.0]) / 3.0
    pe = np.array([1.0, 2.0, 3.0]) + direction * (frac * d)
    e = seg(pe, 0.0, pe, 5.0)
    st, tin, tout, dm = oracle.pair(e, q, d)
    assert st == (1 if hit else 0)
    assert dm == pytest.approx(frac * d, rel=1e-12, abs=1e-12)
    if hit:
        assert (tin, tout) == (2.0, 5.0)


def test_parallel_motion_constant_offset():
    """Equal velocities: the separation is constant, so the pair is in range
    over the whole common span or not at all."""
    v = np.array([0.3, -1.2, 0.7])
    off = np.array([0.0, 4.0, 3.0])  # |off| = 5
    e = moving((10.0, 10.0, 10.0), v, 1.0, 9.0)
    q = moving(np.array([10.0, 10.0, 10.0]) + off, v, 4.0, 12.0)
    st, tin, tout, dm = oracle.pair(e, q, 5.0 + 1e-9)
    assert st == 1 and tin == 4.0 and tout == 9.0
    assert dm == pytest.approx(5.0, rel=1e-12)
    st, *_ = oracle.pair(e, q, 5.0 - 1e-6)
    assert st == 0


@pytest.mark.parametrize("X,u,d,T", [(10.0, 1.0, 2.0, 20.0), (7.5, 0.25, 0.1, 60.0), (3.0, 2.0, 1.0, 1.6)])
def test_head_on_approach(X, u, d, T):
    """Entry x = -X + u t, query x = X - u t on one axis: the separation is
    |2X - 2ut|, in range for t in [(2X - d)/(2u), (2X + d)/(2u)] cut to [0, T]."""
    e = moving((-X, 0.0, 0.0), (u, 0.0, 0.0), 0.0, T)
    q = moving((X, 0.0, 0.0), (-u, 0.0, 0.0), 0.0, T)
    lo = max(0.0, (2 * X - d) / (2 * u))
    hi = min(T, (2 * X + d) / (2 * u))
    st, tin, tout, dm = oracle.pair(e, q, d)
    if lo <= hi:
        assert st == 1
        assert tin == pytest.approx(lo, rel=1e-12, abs=1e-12)
        assert tout == pytest.approx(hi, rel=1e-12, abs=1e-12)
    else:
        assert st == 0
    closest = abs(2 * X - 2 * u * min(T, X / u))
    assert dm == pytest.approx(closest, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("beta,d", [(0.0, 1.0), (0.6, 1.0), (0.999, 1.0), (2.5, 3.0)])
def test_flyby_impact_parameter(beta, d):
    """Relative velocity w, impact parameter beta at time tc: the pair is in
    range for |t - tc| <= sqrt(d^2 - beta^2) / |w|."""
    tc = 5.0
    w = np.array([1.5, 0.0, -2.0])  # |w| = 2.5
    nrm = np.array([0.8, 0.0, 0.6])  # unit, orthogonal to w
    ve = np.array([0.2, 0.4, -0.1])
    pe0 = np.array([3.0, -1.0, 2.0])
    # query position at tc is entry position at tc + beta * nrm
    pq_tc = pe0 + ve * tc + beta * nrm
    vq = ve + w
    pq0 = pq_tc - vq * tc
    e = moving(pe0, ve, 0.0, 10.0)
    q = moving(pq0, vq, 1.0, 11.0)
    half = math.sqrt(d * d - beta * beta) / 2.5
    st, tin, tout, dm = oracle.pair(e, q, d)
    assert st == 1
    assert tin == pytest.approx(tc - half, rel=1e-12)
    assert tout == pytest.approx(tc + half, rel=1e-12)
    assert dm == pytest.approx(beta, abs=1e-12)


def test_touching_spans_are_not_pairs():
    """Consecutive segments that share only an instant have no common span of
    positive length: no pair (strict overlap)."""
    e = seg((0, 0, 0), 0.0, (1, 0, 0), 1.0)
    q = seg((1, 0, 0), 1.0, (2, 0, 0), 2.0)
    assert oracle.pair(e, q, 10.0)[0] == -1
    assert oracle.pair(q, e, 10.0)[0] == -1
    far = seg((0, 0, 0), 5.0, (0, 0, 0), 6.0)
    assert oracle.pair(e, far, 10.0)[0] == -1


def test_window_clips_the_span():
    """The query window [t0, t1] cuts the common span."""
    p = (0.0, 0.0, 0.0)
    e = seg(p, 0.0, p, 10.0)
    q = seg((1.0, 0.0, 0.0), 0.0, (1.0, 0.0, 0.0), 10.0)
    assert oracle.pair(e, q, 2.0, 2.5, 7.25)[:3] == (1, 2.5, 7.25)
    assert oracle.pair(e, q, 2.0, 10.0, 12.0)[0] == -1  # touches only at t = 10
    assert oracle.pair(e, q, 2.0, 7.0, 3.0)[0] == -1  # empty window


def test_exact_crossing_with_zero_threshold():
    """d = 0: segments that pass through the same point at the same time are
    reported with a zero-length interval at that time."""
    e = seg((0, 0, 0), 0.0, (2, 0, 0), 2.0)
    q = seg((2, 0, 0), 0.0, (0, 0, 0), 2.0)
    st, tin, tout, dm = oracle.pair(e, q, 0.0)
    assert (st, tin, tout, dm) == (1, 1.0, 1.0, 0.0)
    q_off = seg((2, 0, 1e-3), 0.0, (0, 0, 1e-3), 2.0)
    assert oracle.pair(e, q_off, 0.0)[0] == 0


def test_identical_segment_is_in_range_over_its_extent():
    """A query segment taken from the database matches itself at distance 0."""
    s = seg((1.0, 2.0, 3.0), 4.0, (2.0, 0.5, 3.5), 5.0)
    assert oracle.pair(s, s, 0.0) == (1, 4.0, 5.0, 0.0)


# --------------------------------------------------------------------------
# Invariants on random pairs
# --------------------------------------------------------------------------

def _random_pairs(rng, n):
    out = []
    for _ in range(n):
        def one():
            t0 = rng.uniform(0, 4)
            t1 = t0 + rng.uniform(0.1, 4)
            return seg(rng.uniform(0, 4, 3), t0, rng.uniform(0, 4, 3), t1)
        out.append((one(), one(), rng.uniform(0.2, 2.5)))
    return out


def test_invariants_on_random_pairs():
    rng = np.random.default_rng(11)
    hits = 0
    for e, q, d in _random_pairs(rng, 3000):
        st, tin, tout, dm = oracle.pair(e, q, d)
        a = max(e[3], q[3])
        b = min(e[7], q[7])
        if st < 0:
            assert not a < b
            continue
        assert a < b
        # symmetric under swapping query and entry
        st2, tin2, tout2, dm2 = oracle.pair(q, e, d)
        assert st2 == st
        assert dm2 == pytest.approx(dm, rel=1e-12, abs=1e-12)
        if st == 0:
            # never in range: sampled distances all exceed d
            ts = np.linspace(a, b, 257)
            assert dist_at(e, q, ts).min() > d * (1 - 1e-9)
            continue
        hits += 1
        assert tin2 == pytest.approx(tin, rel=1e-11, abs=1e-11)
        assert tout2 == pytest.approx(tout, rel=1e-11, abs=1e-11)
        # interval inside the common span
        assert a <= tin <= tout <= b
        # at an endpoint strictly inside the span the separation is exactly d
        for t in (tin, tout):
            dist = dist_at(e, q, t)[0]
            if a < t < b:
                assert dist == pytest.approx(d, rel=1e-9)
            else:
                assert dist <= d * (1 + 1e-9)
        assert dist_at(e, q, 0.5 * (tin + tout))[0] <= d * (1 + 1e-9)
    assert hits > 100


def test_translation_and_scaling_invariance():
    rng = np.random.default_rng(12)
    for e, q, d in _random_pairs(rng, 500):
        base = oracle.pair(e, q, d)
        # translate every position by the same vector
        sh = np.array([100.0, -37.5, 12.25, 0, 100.0, -37.5, 12.25, 0])
        tr = oracle.pair(e + sh, q + sh, d)
        assert tr[0] == base[0] or abs(base[3] - d) <= 1e-9 * d
        if base[0] == 1 and tr[0] == 1:
            assert tr[1] == pytest.approx(base[1], rel=1e-9, abs=1e-9)
            assert tr[2] == pytest.approx(base[2], rel=1e-9, abs=1e-9)
        # scaling every position and d by 2 is exact in binary floating point
        sc = np.array([2, 2, 2, 1, 2, 2, 2, 1.0])
        s2 = oracle.pair(e * sc, q * sc, 2 * d)
        assert s2[0] == base[0]
        if base[0] == 1:
            assert s2[1:3] == base[1:3]


def test_time_shift_invariance():
    """Shifting all times (and the window) by an exactly representable amount,
    with times on a dyadic grid so the shift is exact, shifts the interval."""
    rng = np.random.default_rng(13)
    for e, q, d in _random_pairs(rng, 500):
        for s in (e, q):
            s[3] = np.round(s[3] * 1024) / 1024
            s[7] = s[3] + np.ceil((s[7] - s[3]) * 1024) / 1024
        base = oracle.pair(e, q, d, 0.5, 7.0)
        sh = np.array([0, 0, 0, 256.0, 0, 0, 0, 256.0])
        moved = oracle.pair(e + sh, q + sh, d, 256.5, 263.0)
        assert moved[0] == base[0]
        if base[0] == 1:
            assert moved[1] - 256.0 == pytest.approx(base[1], abs=1e-11)
            assert moved[2] - 256.0 == pytest.approx(base[2], abs=1e-11)


# --------------------------------------------------------------------------
# Dense time sampling on tiny inputs
# --------------------------------------------------------------------------

def test_dense_sampling_agrees_with_intervals():
    """For tiny random sets, sample every common span 10^4 times: samples at
    distance <= d(1-1e-9) lie inside the reported interval, samples at distance
    > d(1+1e-9) lie outside it, and unreported pairs have no sample in range."""
    rng = np.random.default_rng(14)
    ent = workloads.random_segments(rng, 40, box=6.0, t_span=6.0)
    qry = workloads.random_segments(rng, 25, box=6.0, t_span=6.0)
    d = 1.3
    res = oracle.search_bruteforce(ent, qry, d, threads=1)
    reported = {(int(a), int(b)): (x, y) for a, b, x, y in
                zip(res.query_index, res.entry_index, res.t_enter, res.t_exit)}
    checked = 0
    for qi in range(len(qry)):
        q8 = qry.row(qi)
        for ei in range(len(ent)):
            e8 = ent.row(ei)
            a, b = max(e8[3], q8[3]), min(e8[7], q8[7])
            if not a < b:
                assert (qi, ei) not in reported
                continue
            ts = np.linspace(a, b, 10_000)
            dist = dist_at(e8, q8, ts)
            inside_d = dist <= d * (1 - 1e-9)
            outside_d = dist > d * (1 + 1e-9)
            if (qi, ei) in reported:
                tin, tout = reported[(qi, ei)]
                eps = 1e-9 * max(1.0, abs(b))
                inside_t = (ts >= tin - eps) & (ts <= tout + eps)
                assert np.all(inside_t[inside_d])
                strict_in = (ts > tin + eps) & (ts < tout - eps)
                assert not np.any(strict_in & outside_d)
            else:
                assert not np.any(inside_d)
            checked += 1
    assert checked > 50 and len(reported) > 10


# --------------------------------------------------------------------------
# Brute force against the sweep
# --------------------------------------------------------------------------

def _same(r1, r2):
    assert np.array_equal(r1.query_index, r2.query_index)
    assert np.array_equal(r1.entry_index, r2.entry_index)
    assert np.array_equal(r1.t_enter, r2.t_enter)
    assert np.array_equal(r1.t_exit, r2.t_exit)
    assert r1.overlap_pairs == r2.overlap_pairs


def test_bruteforce_equals_sweep_on_random_sets():
    rng = np.random.default_rng(15)
    for k in range(100):
        ent = workloads.random_segments(rng, int(rng.integers(0, 60)), box=5.0, t_span=8.0, max_dur=3.0)
        qry = workloads.random_segments(rng, int(rng.integers(1, 30)), box=5.0, t_span=8.0, max_dur=3.0)
        d = float(rng.uniform(0.0, 2.0))
        t0, t1 = sorted(rng.uniform(-1, 9, 2)) if k % 3 == 0 else (-np.inf, np.inf)
        _same(oracle.search_bruteforce(ent, qry, d, t0, t1, threads=1),
              oracle.search_sweep(ent, qry, d, t0, t1, threads=2))


def test_per_query_sweep_equals_brute_force_per_segment():
    # each query segment with its own d and window: the same pairs and
    # intervals as brute force run segment by segment with those parameters
    rng = np.random.default_rng(16)
    for k in range(40):
        ent = workloads.random_segments(rng, int(rng.integers(0, 60)), box=5.0, t_span=8.0, max_dur=3.0)
        nq = int(rng.integers(1, 20))
        qry = workloads.random_segments(rng, nq, box=5.0, t_span=8.0, max_dur=3.0)
        d = rng.uniform(0.0, 2.0, nq)
        w = np.sort(rng.uniform(-1, 9, (nq, 2)), axis=1)
        if k % 4 == 0:
            w[:, 0], w[:, 1] = -np.inf, np.inf
        got = oracle.search_sweep_per_query(ent, qry, d, w[:, 0], w[:, 1], threads=2)
        parts = [oracle.search_bruteforce(ent, qry.take([i]), d[i], w[i, 0], w[i, 1], threads=1) for i in range(nq)]
        qi = np.concatenate([np.full(len(p.query_index), i, np.int64) for i, p in enumerate(parts)])
        ei = np.concatenate([p.entry_index for p in parts])
        tin = np.concatenate([p.t_enter for p in parts])
        tout = np.concatenate([p.t_exit for p in parts])
        o = np.lexsort((ei, qi))
        assert np.array_equal(got.query_index, qi[o]) and np.array_equal(got.entry_index, ei[o])
        assert np.array_equal(got.t_enter, tin[o]) and np.array_equal(got.t_exit, tout[o])
        assert got.overlap_pairs == sum(p.overlap_pairs for p in parts)


def test_bruteforce_equals_sweep_on_tiny_random_walk():
    w = workloads.tiny_random_walk()
    assert len(w.entries) == 19_800 and len(w.queries) == 20 * 99
    a = oracle.search_bruteforce(w.entries, w.queries, 5.0, *w.window)
    b = oracle.search_sweep(w.entries, w.queries, 5.0, *w.window)
    _same(a, b)
    # time-aligned unit steps: each query segment shares a span with exactly
    # one segment of each of the 200 trajectories
    assert a.overlap_pairs == 20 * 99 * 200
    # every query segment matches itself
    assert len(a.query_index) >= len(w.queries)


# --------------------------------------------------------------------------
# The index example of Sec. 4
# --------------------------------------------------------------------------

def test_fig1_bin_table():
    g = read_golden("fig1_bins.txt")
    segs = np.array(g["segments"])
    bt = oracle.bin_table(segs[:, 1], segs[:, 2], 4)
    assert bt["width"] == 3.0
    assert np.array_equal(bt["order"], segs[:, 0].astype(np.int64))
    for j, bstart, bend, bfirst, blast in g["bins"]:
        j = int(j)
        assert bt["start"][j] == bstart
        assert bt["end"][j] == bend
        assert bt["first"][j] == int(bfirst)
        assert bt["last"][j] == int(blast)


def test_fig1_bin_table_time_shifted():
    """Fig. 1 with every time shifted by 1000: the same bins (the extent now
    starts at 1000), the same index ranges, extents shifted by 1000."""
    g = read_golden("fig1_bins.txt")
    segs = np.array(g["segments"])
    bt = oracle.bin_table(1000.0 + segs[:, 1], 1000.0 + segs[:, 2], 4)
    assert bt["width"] == 3.0
    for j, bstart, bend, bfirst, blast in g["bins"]:
        j = int(j)
        assert bt["start"][j] == 1000.0 + bstart
        assert bt["end"][j] == 1000.0 + bend
        assert (bt["first"][j], bt["last"][j]) == (int(bfirst), int(blast))


def test_fig2_batch_interactions_documented_mismatch():
    """Fig. 2's printed totals cannot all be reproduced under one reading of the
    bin extent: the text defines B_start = j*b, the figure prints the smallest
    t_start.  The computed totals under both readings are recorded here; only
    some agree with the printed ones (450, 600, 630, 900)."""
    g1 = read_golden("fig1_bins.txt")
    g2 = read_golden("fig2_batches.txt")
    segs = np.array(g1["segments"])
    bt = oracle.bin_table(segs[:, 1], segs[:, 2], 4)
    batches = np.array(g2["batches"])
    printed = {int(s): int(t) for s, t in g2["printed"]}
    jb = np.arange(4) * bt["width"]

    def totals(lo):
        out = {}
        for size in (10, 20, 30, 60):
            k = size // 10
            cnt, bts, bte = [], [], []
            for i in range(0, 6, k):
                grp = batches[i:i + k]
                cnt.append(int(grp[:, 0].sum()))
                bts.append(grp[:, 1].min())
                bte.append(grp[:, 2].max())
            out[size] = oracle.batch_interactions(lo, bt["end"], bt["first"], bt["last"], cnt, bts, bte)
        return out

    t_min = totals(bt["start"])
    t_jb = totals(jb)
    assert t_min == {10: 420, 20: 540, 30: 540, 60: 900}
    assert t_jb == {10: 510, 20: 660, 30: 630, 60: 900}
    assert printed == {10: 450, 20: 600, 30: 630, 60: 900}
    # the all-in-one batch (60 segments against all 15 entries) agrees everywhere
    assert t_min[60] == t_jb[60] == printed[60] == 60 * 15


# --------------------------------------------------------------------------
# Self-join (query (ii) of Sec. 2.1 with the database as the query set)
# --------------------------------------------------------------------------

def _segments_from_rows(rows, traj, seg_ids):
    rows = np.asarray(rows, np.float64)
    return workloads.Segments(*[rows[:, k].copy() for k in range(8)], np.asarray(seg_ids, np.int64),
                              np.asarray(traj, np.int64))


def test_self_join_head_on_pair_once():
    """Two one-segment trajectories approaching head-on, and a second segment
    of the first trajectory lying on top of the first: the self-join reports
    the head-on pair once, with the closed-form interval, and never the pair
    of one trajectory."""
    X, u, d, T = 10.0, 2.0, 3.0, 10.0
    rows = [moving((-X, 0, 0), (u, 0, 0), 0.0, T), moving((X, 0, 0), (-u, 0, 0), 0.0, T),
            moving((-X, 0, 0), (u, 0, 0), 0.0, T)]
    ent = _segments_from_rows(rows, traj=[7, 9, 7], seg_ids=[5, 3, 8])
    r = oracle.self_join(ent, d)
    # unordered pairs of different trajectories: (5,3) and (8,3); reported with the smaller id as the query
    got = sorted((int(ent.seg_id[q]), int(ent.seg_id[e])) for q, e in zip(r.query_index, r.entry_index))
    assert got == [(3, 5), (3, 8)]
    lo, hi = (2 * X - d) / (2 * u), (2 * X + d) / (2 * u)
    assert np.allclose(r.t_enter, lo, rtol=1e-12) and np.allclose(r.t_exit, hi, rtol=1e-12)
    # the overlap count covers every ordered pair, the left-out ones included
    assert r.overlap_pairs == 9


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_self_join_is_the_filtered_full_search(seed):
    """The self-join equals the full search of the database against itself
    with the pairs of one trajectory removed and, of the two orders of a
    pair, the one whose entry id is larger kept; the removed order carries
    the same interval (swap symmetry), so nothing is lost."""
    w = workloads.tiny_random_walk(seed=seed, n_traj=60, n_points=30)
    ent = w.entries
    perm = np.random.default_rng(seed).permutation(len(ent))
    ent.seg_id = ent.seg_id[perm]  # ids unrelated to positions
    d = 12.0
    sj = oracle.self_join(ent, d)
    full = oracle.search_sweep(ent, ent, d)
    assert sj.overlap_pairs == full.overlap_pairs
    other = ent.traj_id[full.query_index] != ent.traj_id[full.entry_index]
    keep = other & (ent.seg_id[full.entry_index] > ent.seg_id[full.query_index])
    key = lambda qi, ei: list(zip(qi.tolist(), ei.tolist()))  # noqa: E731
    assert key(sj.query_index, sj.entry_index) == key(full.query_index[keep], full.entry_index[keep])
    assert np.array_equal(sj.t_enter, full.t_enter[keep]) and np.array_equal(sj.t_exit, full.t_exit[keep])
    # swap symmetry: every dropped order of a cross-trajectory pair is the
    # reverse of a kept one with the same interval
    rev = {(e, q): (a, b) for q, e, a, b in zip(full.query_index[keep], full.entry_index[keep],
                                                 full.t_enter[keep], full.t_exit[keep])}
    dropped = other & ~keep
    assert int(dropped.sum()) == int(keep.sum()) > 0
    for q, e, a, b in zip(full.query_index[dropped], full.entry_index[dropped], full.t_enter[dropped],
                          full.t_exit[dropped]):
        ra, rb = rev[(q, e)]
        assert ra == pytest.approx(a, rel=1e-12, abs=1e-12) and rb == pytest.approx(b, rel=1e-12, abs=1e-12)
