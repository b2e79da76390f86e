"""The temporal bins of Sec. 4 at their boundaries.  The search finds the
bin of a query segment's clipped start and end exactly -- its exact count of
temporal-overlap pairs and the end of its candidate range are searched
inside those bins of the sorted keys -- from a table of each bin's smallest
time key (built with the index from the bin function floor((t - t_min) / b)
itself) rather than by dividing.  Query spans that start and end within a
few ulps of bin boundaries, for several bin counts and an awkward t_min,
and entries that all start at one instant, must give the oracle's overlap
counts and pairs."""
import numpy as np
import pytest

from oracle import oracle
from paper_1405_7461_gb300 import workloads

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


def _bin(t, t_min, width, m):
    # the bin function of the index (numpy: IEEE division and floor)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.floor((np.float64(t) - t_min) / width)
    if not f < m - 1:
        return m - 1
    return 0 if f < 0 else int(f)


def _boundary(b, t_min, width, m):
    # smallest double whose bin is >= b (b >= 1), near t_min + b width;
    # bin 0 is taken to start at t_min
    if b <= 0:
        return np.float64(t_min)
    t = np.float64(t_min + b * width)
    for _ in range(64):
        if _bin(t, t_min, width, m) < b:
            break
        t = np.nextafter(t, -np.inf)
    else:
        raise AssertionError("no boundary below")
    for _ in range(128):
        if _bin(t, t_min, width, m) >= b:
            return t
        t = np.nextafter(t, np.inf)
    raise AssertionError("no boundary above")


def _segs(ts, te, rng, first_id=0):
    n = len(ts)
    p0 = rng.uniform(0.0, 5.0, (n, 3))
    p1 = p0 + rng.normal(0.0, 0.5, (n, 3))
    return workloads.Segments.from_columns([p0[:, 0], p0[:, 1], p0[:, 2], ts, p1[:, 0], p1[:, 1], p1[:, 2], te],
                                           seg_id=np.arange(first_id, first_id + n))


def _check(tdq, ent, qry, m, d=2.0):
    with tdq.build_index(ent, bin_count=m) as idx:
        r = tdq.search(idx, qry, d, mode=tdq.MODE_FP32_FILTER)
        st = tdq.get_stats(idx)
        r64 = tdq.search(idx, qry, d, mode=tdq.MODE_FP64)
    ref = oracle.search_sweep(ent, qry, d)
    assert st["overlap_pairs"] == ref.overlap_pairs
    for res in (r, r64):
        got = set(zip(res.query_seg_id.tolist(), res.entry_seg_id.tolist()))
        want = set(zip(qry.seg_id[ref.query_index].tolist(), ent.seg_id[ref.entry_index].tolist()))
        assert got == want


@pytest.mark.parametrize("m", [1, 3, 7, 1000, 100_000])
def test_query_spans_at_bin_boundaries(tdq, m):
    rng = np.random.default_rng(m)
    # entries: start times in [0.1, 0.1 + 37.3] (t_min 0.1: no exact width)
    n = 6000
    ts = 0.1 + 37.3 * rng.random(n)
    ts[0], ts[1] = 0.1, 37.4
    te = ts + rng.uniform(0.01, 1.5, n)
    ent = _segs(ts, te, rng)
    # the index's extent: the first entry start to the last entry end
    t_min, t_max = float(ts.min()), float(te.max())
    width = (t_max - t_min) / m
    # query spans from one boundary (+- a few ulps) to another
    bs = rng.integers(0, m, 300) if m > 1 else np.zeros(300, np.int64)
    q0, q1 = [], []
    for k, b in enumerate(bs):
        t = _boundary(int(b), t_min, width, m) if b > 0 else np.float64(t_min)
        for _ in range(int(rng.integers(-3, 4))):
            t = np.nextafter(t, np.inf if k % 2 else -np.inf)
        e = _boundary(int(min(m - 1, b + rng.integers(0, 3))), t_min, width, m) if m > 1 else np.float64(t_max)
        for _ in range(int(rng.integers(0, 4))):
            e = np.nextafter(e, np.inf)
        if not e > t:
            e = t + 0.25
        q0.append(t)
        q1.append(e)
    qry = _segs(np.array(q0), np.array(q1), rng, first_id=10 ** 6)
    _check(tdq, ent, qry, m)


def test_entries_starting_at_one_instant(tdq):
    # every entry starts at the same time: all of them in bin 0, query spans
    # at, just before and just after that instant
    rng = np.random.default_rng(9)
    n = 3000
    ts = np.full(n, 5.0)
    te = ts + rng.uniform(0.1, 3.0, n)
    ent = _segs(ts, te, rng)
    q0 = np.concatenate([np.array([4.0, 5.0, np.nextafter(5.0, 0.0), np.nextafter(5.0, 9.0)]), rng.uniform(3.0, 8.0, 60)])
    qry = _segs(q0, q0 + rng.uniform(0.05, 2.0, len(q0)), rng, first_id=10 ** 6)
    for m in (1, 64, 10_000):
        _check(tdq, ent, qry, m)
