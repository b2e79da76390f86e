"""Failure detection without a GPU fault: every allocation of a full
scenario (index build, searches in both modes, a batched plan, a server) is
made to fail in turn on the host side; each call must report TDQ_ERR_NOMEM
or succeed, the library must stay usable, and no device memory may leak."""
import numpy as np
import pytest

from paper_1405_7461_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _scenario(tdq, ent, q):
    """Runs until the first failure; returns the status of the failing call
    (TDQ_OK if none failed)."""
    objs = []
    try:
        idx = tdq.build_index(ent, bin_count=500)
        objs.append(idx)
        tdq.search(idx, q, 2.0)
        tdq.search(idx, q, 2.0, mode=tdq.MODE_FP32_FILTER)
        plan = tdq.Plan(idx, len(q), mode=tdq.MODE_FP32_FILTER)
        objs.append(plan)
        n = len(q)
        plan.search(q, np.full(n, 2.0), np.full(n, -np.inf), np.full(n, np.inf))
        srv = tdq.Server(idx, max_batch_query_segments=1024, lanes=2)
        objs.append(srv)
        srv.wait(srv.submit(q, 2.0, -np.inf, np.inf))
        return tdq.TDQ_OK
    except tdq.TdqError as e:
        return e.status
    finally:
        for o in reversed(objs):
            o.free()


def test_every_allocation_failure_is_reported_without_leaks(tdq_lib=None):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7461_gb300 import build, tdq

    build.build()
    tdq.load()
    rng = np.random.default_rng(31)
    ent = workloads.random_segments(rng, 4000, box=10.0, t_span=20.0)
    q = workloads.random_segments(rng, 300, box=10.0, t_span=20.0)
    tdq.debug_fail_allocations(-1)
    assert _scenario(tdq, ent, q) == tdq.TDQ_OK  # warm: module loading, driver pools
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    statuses = []
    k = 0
    try:
        while True:
            tdq.debug_fail_allocations(k)
            st = _scenario(tdq, ent, q)
            statuses.append(st)
            assert st in (tdq.TDQ_OK, tdq.TDQ_ERR_NOMEM), (k, st, tdq.last_error())
            if st == tdq.TDQ_OK:
                break  # the scenario made fewer than k + 1 allocations
            k += 1
            assert k < 400
    finally:
        tdq.debug_fail_allocations(-1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert statuses.count(tdq.TDQ_ERR_NOMEM) >= 15
    # and the library still works
    assert _scenario(tdq, ent, q) == tdq.TDQ_OK
