"""The allocation-free search entry point (tdq_search_device_noalloc).

Some callers cannot allocate device memory when they search: their device
memory is owned by another allocator, or they run a latency-critical loop
that cannot afford cudaMalloc/cudaFree (which may synchronize the device).
For them the library keeps the per-search scratch in one fixed device array.
This file checks, through the C ABI, that two calls in a row return the same
results as tdq_search_device (pair sets equal, endpoints within the parity
tolerance), that the fixed size limit is enforced with a clear error, and
that a call does not change the device's free memory.  It is named so that
pytest collects it last."""
import numpy as np
import pytest

from paper_1405_7461_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ENDPOINT_REL = 1e-9


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


def _same(a, b):
    qa, ea, ia, xa = _sorted(a)
    qb, eb, ib, xb = _sorted(b)
    assert np.array_equal(qa, qb) and np.array_equal(ea, eb)
    assert np.all(np.abs(ia - ib) <= ENDPOINT_REL * np.maximum(1.0, np.abs(ib)))
    assert np.all(np.abs(xa - xb) <= ENDPOINT_REL * np.maximum(1.0, np.abs(xb)))


def test_noalloc_matches_device_search_on_two_calls(tdq):
    w = workloads.scale_random_walk(n_traj=1200, n_queries=9, seed=77)
    nq = len(w.queries)
    assert 32 < nq <= tdq.NOALLOC_MAX_QUERIES and nq % 32 != 0  # several tiles and a ragged tail
    with tdq.build_index(w.entries) as idx:
        qdev = tdq.DeviceSegments(w.queries)
        ref_buf = tdq.DeviceResultBuffer(1 << 16)
        buf = tdq.DeviceResultBuffer(1 << 16)
        for d in (15.0, 5.0):  # two calls in a row, the second after the first filled the scratch
            n_ref = tdq.search_device(idx, qdev, d, *w.window, ref_buf)
            ref = ref_buf.to_host(n_ref)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            n = tdq.search_device_noalloc(idx, qdev, d, *w.window, buf)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            assert free_after == free_before
            assert n == n_ref >= len(w.queries)  # every query segment matches itself
            _same(buf.to_host(n), ref)


def test_noalloc_rejects_more_than_the_limit(tdq):
    rng = np.random.default_rng(3)
    ent = workloads.random_segments(rng, 100)
    too_many = workloads.random_segments(rng, tdq.NOALLOC_MAX_QUERIES + 1)
    with tdq.build_index(ent) as idx:
        buf = tdq.DeviceResultBuffer(16)
        with pytest.raises(tdq.TdqError) as ei:
            tdq.search_device_noalloc(idx, tdq.DeviceSegments(too_many), 1.0, -np.inf, np.inf, buf)
        assert ei.value.status == tdq.TDQ_ERR_INVALID
        assert "8192" in str(ei.value)
        # an in-limit call still works afterwards
        ok = workloads.random_segments(rng, 50)
        n = tdq.search_device_noalloc(idx, tdq.DeviceSegments(ok), 1.0, -np.inf, np.inf, buf,
                                      allow_overflow=True)
        assert n >= 0


def test_noalloc_accepts_only_the_plain_fp64_mode(tdq):
    # the filter mode's survivor list has no fixed bound, and the pair
    # filters belong to the self-join: both are refused with a message
    rng = np.random.default_rng(4)
    ent = workloads.random_segments(rng, 200)
    q = tdq.DeviceSegments(workloads.random_segments(rng, 40))
    with tdq.build_index(ent) as idx:
        buf = tdq.DeviceResultBuffer(1 << 12)
        with pytest.raises(tdq.TdqError) as ei:
            tdq.search_device_noalloc(idx, q, 1.0, -np.inf, np.inf, buf, mode=tdq.MODE_FP32_FILTER)
        assert ei.value.status == tdq.TDQ_ERR_INVALID and "TDQ_MODE_FP64" in str(ei.value)
        with pytest.raises(tdq.TdqError) as ei:
            tdq.search_device_noalloc(idx, q, 1.0, -np.inf, np.inf, buf, flags=tdq.FLAG_OTHER_TRAJECTORIES)
        assert ei.value.status == tdq.TDQ_ERR_INVALID and "flags" in str(ei.value)
        # the plain mode still runs after the refusals
        assert tdq.search_device_noalloc(idx, q, 1.0, -np.inf, np.inf, buf, mode=tdq.MODE_FP64,
                                         allow_overflow=True) >= 0
