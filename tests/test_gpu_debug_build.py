"""The bounds-checked debug build (libtdq_debug.so, compiled with
-DTDQ_DEBUG), the GPU counterpart of a memory checker.  Every index the
search kernels compute before an access -- tile and candidate ranges,
sorted positions, prefetched passes, survivor and result slots, tensor-core
record blocks -- is checked against its bounds; a failed check skips the
access and makes the search fail with TDQ_ERR_CUDA naming the site.  This
test builds the variant and, in a fresh process that loads it, runs the tiny
workload and a reduced scale walk through every mode (plain FP64, FP32
pre-test, tensor-core pre-test), a batched plan, a self-join and the
allocation-free call, each checked against the oracle or the plain mode: no
check may fail (Sec. 5 sizes the result buffer; overflow is a separate,
reported status)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_1405_7461_gb300 import build, tdq, workloads
from oracle import oracle
from tests._util import compare_results
lib = tdq.load(build.build(debug=True))
assert "debug" in tdq.version(), tdq.version()
import torch

def positions(ids, pool):
    o = np.argsort(pool, kind="stable")
    return o[np.searchsorted(pool[o], ids)]

def sorted_arrays(r):
    o = np.lexsort((r.entry_seg_id, r.query_seg_id))
    return r.query_seg_id[o], r.entry_seg_id[o], r.t_enter[o], r.t_exit[o]

checked = 0
for w, brute in ((workloads.tiny_random_walk(), True), (workloads.scale_random_walk(n_traj=1500, n_queries=12), False)):
    with tdq.build_index(w.entries) as idx:
        for d in w.d_values:
            ref = (oracle.search_bruteforce if brute else oracle.search_sweep)(w.entries, w.queries, d, *w.window)
            base = None
            for mode in (tdq.MODE_FP64, tdq.MODE_FP32_FILTER, tdq.MODE_TC_FILTER):
                r = tdq.search(idx, w.queries, d, *w.window, mode=mode)
                if base is None:
                    base = r
                    got = {"qi": positions(r.query_seg_id, w.queries.seg_id),
                           "ei": positions(r.entry_seg_id, w.entries.seg_id), "t_enter": r.t_enter,
                           "t_exit": r.t_exit}
                    cmp = compare_results(got, {"qi": ref.query_index, "ei": ref.entry_index,
                                                "t_enter": ref.t_enter, "t_exit": ref.t_exit},
                                          w.entries, w.queries, d, *w.window,
                                          dmin_fn=lambda ei, qi: oracle.pair_dmin(w.entries, ei, w.queries, qi,
                                                                                 *w.window))
                    assert cmp["matched"] == len(ref.query_index)
                else:
                    for a, b in zip(sorted_arrays(base), sorted_arrays(r)):
                        assert np.array_equal(a, b)
                checked += 1
        # a batched plan (graph replay) with per-segment d, and the allocation-free call
        q = w.queries
        n = len(q)
        with tdq.Plan(idx, n, mode=tdq.MODE_FP32_FILTER) as plan:
            plan.search(q, np.full(n, w.d_values[-1]), np.full(n, w.window[0]), np.full(n, w.window[1]))
            pr = plan.results()
        for a, b in zip(sorted_arrays(pr), sorted_arrays(tdq.search(idx, q, w.d_values[-1], *w.window))):
            assert np.array_equal(a, b)
        if n <= tdq.NOALLOC_MAX_QUERIES:
            buf = tdq.DeviceResultBuffer(1 << 16)
            c = tdq.search_device_noalloc(idx, tdq.DeviceSegments(q), w.d_values[0], *w.window, buf)
            assert c == len(tdq.search(idx, q, w.d_values[0], *w.window))
        checked += 2
# self-join (pair filters) in both pre-test modes
w = workloads.tiny_random_walk(n_traj=100, n_points=50)
with tdq.build_index(w.entries) as idx:
    a = tdq.self_join(idx, w.entries, 4.0, mode=tdq.MODE_FP32_FILTER)
    b = tdq.self_join(idx, w.entries, 4.0, mode=tdq.MODE_TC_FILTER)
    for x, y in zip(sorted_arrays(a), sorted_arrays(b)):
        assert np.array_equal(x, y)
    checked += 2
print("DEBUG_BUILD_OK", checked)
'''


def test_debug_build_runs_every_mode_with_no_failed_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    code = "ROOT = %r\n" % ROOT + CHILD
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "DEBUG_BUILD_OK" in r.stdout
