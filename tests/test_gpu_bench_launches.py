"""The benchmark's own timed launches against the oracle, at full size.

The headline step of bench.py is one filter-mode plan over the default
scale random-walk workload (10,000 walks, 2.49 M entry segments, 100 query
trajectories) with the three thresholds d in {1, 5, 15} concatenated into one
batch of per-segment d; its end-to-end leg runs the same batch from pinned
host arrays through a plan with host_results.  Both are built here by the
bench's own functions (bench.workload, bench.concat_thresholds,
bench.headline_plan, bench.pinned_queries), so the settings cannot drift,
and every pair of every threshold is compared with the time-sweep oracle
(Sec. 4: one lookup over the whole query set; Sec. 6.1: a fixed batch)."""
import numpy as np
import pytest

from oracle import oracle
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


def _per_threshold(res, w, k_thresholds):
    """Split a batched result by threshold (the bench tags copy k of the
    query set with seg_id + k << 40) into oracle-index form."""
    k = res.query_seg_id >> 40
    base = res.query_seg_id & ((1 << 40) - 1)
    qo = np.argsort(w.queries.seg_id, kind="stable")
    eo = np.argsort(w.entries.seg_id, kind="stable")
    out = []
    for j in range(k_thresholds):
        m = k == j
        qi = qo[np.searchsorted(w.queries.seg_id[qo], base[m])]
        ei = eo[np.searchsorted(w.entries.seg_id[eo], res.entry_seg_id[m])]
        assert np.all(w.queries.seg_id[qi] == base[m]) and np.all(w.entries.seg_id[ei] == res.entry_seg_id[m])
        out.append({"qi": qi, "ei": ei, "t_enter": res.t_enter[m], "t_exit": res.t_exit[m]})
    assert np.all((k >= 0) & (k < k_thresholds))
    return out


def test_headline_and_e2e_launches_match_the_oracle(tdq):
    import bench

    args = bench.parse([])
    w = bench.workload(args, 0)
    assert len(w.entries) > 2_000_000 and args.n_queries == 100
    q3, d3, t03, t13 = bench.concat_thresholds(w)
    nd = len(w.d_values)
    idx = tdq.build_index(tdq.DeviceSegments(w.entries))
    try:
        # the headline: device inputs, device results
        plan = bench.headline_plan(tdq, idx, len(q3))
        cnt = plan.search(tdq.DeviceSegments(q3), *(torch.from_numpy(a).cuda() for a in (d3, t03, t13)))
        head = plan.results()
        st = plan.stats()
        plan.free()
        assert cnt == len(head)
        # the end-to-end leg: pinned host inputs, results in page-locked host memory
        eplan = bench.headline_plan(tdq, idx, len(q3), host_results=True)
        qh, dh, t0h, t1h = bench.pinned_queries(tdq, torch, q3, d3, t03, t13)
        ecnt = eplan.search(qh, dh, t0h, t1h)
        v = eplan.results(view=True)  # as the bench reads them: in the plan's page-locked buffer
        e2e = tdq.Results(*(np.array(getattr(v, f)) for f in ("query_seg_id", "entry_seg_id", "t_enter",
                                                               "t_exit")))
        del v
        est = eplan.stats()
        eplan.free()
        assert ecnt == len(e2e) == cnt
        assert est["overlap_pairs"] == st["overlap_pairs"]
    finally:
        idx.free()
    ora_overlap = 0
    for res, name in ((head, "headline"), (e2e, "e2e")):
        parts = _per_threshold(res, w, nd)
        for j, d in enumerate(w.d_values):
            ref = oracle.search_sweep(w.entries, w.queries, d, *w.window)
            if name == "headline":
                ora_overlap += ref.overlap_pairs
            cmp = compare_results(parts[j], {"qi": ref.query_index, "ei": ref.entry_index, "t_enter": ref.t_enter,
                                             "t_exit": ref.t_exit}, w.entries, w.queries, d, *w.window,
                                  dmin_fn=lambda ei, qi: oracle.pair_dmin(w.entries, ei, w.queries, qi, *w.window))
            assert cmp["matched"] == len(ref.query_index) > 0, (name, d, cmp)
    # the benchmark's unit of work is exact integer work: equal to the oracle's
    assert st["overlap_pairs"] == ora_overlap
