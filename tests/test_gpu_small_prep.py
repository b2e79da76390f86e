"""The two preparations of a search (Sec. 4: clip, sort Q by start, look up
the candidate ranges, plan the tiles).  Up to 1,024 query slots one launch
prepares the whole search (query_prep_small: blocks prepare the slots, the
last one sorts the valid segments by temporal bin in shared memory -- or
finds them in order already -- and plans the tiles); above that the
multi-block chain does (query_prep, the counting sort's scatter,
query_gather).  The same queries
sent through either must give bitwise the same pairs and intervals, and the
oracle's (Sec. 3 / Algorithm 1)."""
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
def entries():
    rng = np.random.default_rng(77)
    return workloads.random_segments(rng, 20_000, box=40.0, t_span=30.0, max_dur=2.0)


def _sorted(r):
    o = np.lexsort((r.entry_seg_id, r.query_seg_id))
    return r.query_seg_id[o], r.entry_seg_id[o], r.t_enter[o], r.t_exit[o]


def _queries(n, seed, time_order=False):
    rng = np.random.default_rng(seed)
    q = workloads.random_segments(rng, n, box=40.0, t_span=30.0, max_dur=2.0)
    if time_order:  # slots in start-time order, as a request's segments come (no sort needed)
        q = q.take(np.argsort(q.ts, kind="stable"))
    q.seg_id = np.arange(n, dtype=np.int64) + 10 ** 6
    d = rng.uniform(0.5, 4.0, n)
    t0 = rng.uniform(-1.0, 12.0, n)
    t1 = t0 + rng.uniform(0.0, 25.0, n)
    t1[::7] = t0[::7]  # empty windows: invalid for the sort, no pairs
    return q, d, t0, t1


@pytest.mark.parametrize("order", ["shuffled", "time"])
@pytest.mark.parametrize("mode_name", ["fp64", "fp32filter"])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 128, 129, 500, 700, 1023, 1024, 1025])
def test_one_block_and_multi_block_preparation_agree(tdq, entries, n, mode_name, order):
    mode = {"fp64": tdq.MODE_FP64, "fp32filter": tdq.MODE_FP32_FILTER}[mode_name]
    q, d, t0, t1 = _queries(n, 900 + n, time_order=order == "time")
    # the same batch followed by 2,048 segments with empty windows (neither
    # errors nor valid segments: they take part in no pair), which puts it
    # above one block's 1,024 slots
    pad = 2048
    dummy = _queries(pad, 1)[0]
    dummy.seg_id = dummy.seg_id + 5 * 10 ** 6
    qb = workloads.Segments.from_columns([np.concatenate([getattr(q, c), getattr(dummy, c)])
                                          for c in workloads.COLUMNS],
                                         seg_id=np.concatenate([q.seg_id, dummy.seg_id]))
    db = np.concatenate([d, np.ones(pad)])
    t0b = np.concatenate([t0, np.zeros(pad)])
    t1b = np.concatenate([t1, np.zeros(pad)])
    with tdq.build_index(entries) as idx:
        with tdq.Plan(idx, n, mode, result_capacity=1 << 16) as ps, \
                tdq.Plan(idx, n + pad, mode, result_capacity=1 << 16) as pl:
            ps.search(q, d, t0, t1)
            rs, ss = ps.results(), ps.stats()
            pl.search(qb, db, t0b, t1b)
            rl, sl = pl.results(), pl.stats()
    for a, b in zip(_sorted(rs), _sorted(rl)):
        assert np.array_equal(a, b)
    for k in ("query_segments", "overlap_pairs", "results"):
        assert ss[k] == sl[k], k
    # one launch prepares a batch of at most 1,024 slots: query_prep_small,
    # then the pair kernel (filter mode: the pre-test, which refines its own
    # survivors)
    if n <= 1024:
        assert ss["kernel_launches"] == 2
    assert sl["kernel_launches"] > 2
    ref = oracle.search_sweep_per_query(entries, q, d, t0, t1)
    qo = np.argsort(q.seg_id)
    got = {"qi": qo[np.searchsorted(q.seg_id[qo], rs.query_seg_id)], "ei": rs.entry_seg_id.copy(),
           "t_enter": rs.t_enter, "t_exit": rs.t_exit}
    cmp = compare_results(got, {"qi": ref.query_index, "ei": ref.entry_index, "t_enter": ref.t_enter,
                                "t_exit": ref.t_exit}, entries, q, 0.0,
                          dmin_fn=lambda ei, qi: oracle.pair_dmin(entries, ei, q, qi), d_per_query=d,
                          win_per_query=(t0, t1))
    assert cmp["matched"] == len(ref.query_index)


def test_one_block_preparation_reports_invalid_input(tdq, entries):
    q, d, t0, t1 = _queries(300, 5)
    q.xs[17] = np.nan
    with tdq.build_index(entries) as idx:
        with pytest.raises(tdq.TdqError) as ei:
            tdq.search(idx, q, 1.0)
        assert ei.value.status == tdq.TDQ_ERR_INVALID
        # the next search (counters cleared by the kernel itself) is clean
        q2, _, _, _ = _queries(300, 6)
        r = tdq.search(idx, q2, 1.0)
        ref = oracle.search_sweep(entries, q2, 1.0)
        assert len(r) == len(ref.query_index)


def test_one_block_preparation_with_all_segments_outside_the_window(tdq, entries):
    q, _, _, _ = _queries(200, 8)
    with tdq.build_index(entries) as idx:
        r = tdq.search(idx, q, 3.0, 1000.0, 2000.0)
        st = tdq.get_stats(idx)
    assert len(r) == 0
    assert st["query_segments"] == 0 and st["work_items"] == 0
