"""CPU-side checks: the C library loads and exports every symbol the header
declares, the product package never touches the oracle, and the workload
generators produce what their docstrings state."""
import ast
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1405_7461_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tdq.h")
PKG = os.path.join(ROOT, "paper_1405_7461_gb300")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdq_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1405_7461_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("tdq_build_index", "tdq_search", "tdq_search_device", "tdq_results_free", "tdq_index_free",
                 "tdq_get_stats", "tdq_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in tdq.h but not exported"


def test_binding_covers_every_declared_symbol():
    from paper_1405_7461_gb300 import tdq

    assert sorted(tdq.SIGNATURES) == declared_functions()


def test_version_and_error_calls_need_no_gpu(lib):
    from paper_1405_7461_gb300 import tdq

    tdq.load()
    assert "sm_103a" in tdq.version()
    assert isinstance(tdq.last_error(), str)


def test_product_package_does_not_import_the_oracle():
    for fn in os.listdir(PKG):
        if not fn.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(PKG, fn)).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert all(not a.name.startswith("oracle") for a in node.names), fn
            if isinstance(node, ast.ImportFrom):
                assert not (node.module or "").startswith("oracle"), fn
    for fn in os.listdir(os.path.join(PKG, "csrc")):
        src = open(os.path.join(PKG, "csrc", fn)).read()
        assert "oracle" not in src.lower(), fn


def test_missing_library_fails_loudly(tmp_path):
    from paper_1405_7461_gb300 import tdq

    saved = tdq._lib
    tdq._lib = None
    try:
        with pytest.raises(RuntimeError):
            tdq.load(str(tmp_path / "nope.so"))
    finally:
        tdq._lib = saved


# --------------------------------------------------------------------------
# Generators
# --------------------------------------------------------------------------

def _check_polylines(seg):
    assert np.all(seg.te > seg.ts)
    same = seg.traj_id[1:] == seg.traj_id[:-1]
    # consecutive segments of one trajectory share their endpoint exactly
    for a, b in (("xe", "xs"), ("ye", "ys"), ("ze", "zs"), ("te", "ts")):
        assert np.array_equal(getattr(seg, a)[:-1][same], getattr(seg, b)[1:][same])
    assert np.all(np.diff(seg.seg_id) > 0)


def test_tiny_random_walk_shape():
    w = workloads.tiny_random_walk()
    e = w.entries
    assert len(e) == 200 * 99
    _check_polylines(e)
    assert e.ts.min() == 0.0 and e.te.max() == 99.0
    assert np.all(e.te - e.ts == 1.0)
    assert len(np.unique(w.queries.traj_id)) == 20
    assert w.window == (0.0, 99.0) and w.d_values == (5.0,)


def test_scale_random_walk_shape_small():
    w = workloads.scale_random_walk(n_traj=300, n_queries=7)
    e = w.entries
    _check_polylines(e)
    counts = np.bincount(e.traj_id)
    assert counts.min() >= 99 and counts.max() <= 399
    starts = np.array([e.ts[e.traj_id == k].min() for k in range(300)])
    assert starts.min() >= 0 and starts.max() <= 200
    assert len(np.unique(w.queries.traj_id)) == 7


def test_galaxy_disk_shape_small():
    w = workloads.galaxy_disk(n_stars=200, n_queries=5)
    e = w.entries
    _check_polylines(e)
    assert len(e) == 200 * 199
    r = np.hypot(e.xs, e.ys)
    assert r.min() >= 0.5 - 1e-12 and r.max() <= 15.0 + 1e-12
    speed = np.sqrt((e.xe - e.xs) ** 2 + (e.ye - e.ys) ** 2)
    # about 220 km/s in kpc per Myr, with 10% dispersion
    assert 0.15 < np.median(speed) < 0.3


def test_batching_walks_shape_small():
    w = workloads.batching_walks(n_traj=100, n_queries=50)
    _check_polylines(w.entries)
    _check_polylines(w.queries)
    nseg = w.meta["query_traj_segments"]
    assert nseg.min() >= 10 and nseg.max() <= 299
    assert len(w.q_d) == len(w.queries)
    assert np.all((w.q_d >= 0.5) & (w.q_d <= 10.0))
    assert np.all(w.q_t0 <= w.q_t1)
    assert np.all(w.queries.te <= 299.0)


def test_host_results_are_views_released_with_their_last_array(monkeypatch):
    # library-owned host results reach Python as views of the library's own
    # arrays (no copy); the block goes back through tdq_results_free exactly
    # once, after the last of the four arrays is gone
    import gc

    from paper_1405_7461_gb300 import tdq

    cols = [np.arange(5, dtype=np.int64) + 100, np.arange(5, dtype=np.int64) + 200,
            np.linspace(0.0, 1.0, 5), np.linspace(2.0, 3.0, 5)]
    r = tdq.tdq_results(cols[0].ctypes.data, cols[1].ctypes.data, cols[2].ctypes.data, cols[3].ctypes.data, 5)
    ptr = ctypes.pointer(r)
    freed = []

    class FakeLib:
        def tdq_results_free(self, p):
            freed.append(ctypes.addressof(p.contents))

    monkeypatch.setattr(tdq, "_lib", FakeLib())
    res = tdq._take_results(ptr)
    for got, want in zip((res.query_seg_id, res.entry_seg_id, res.t_enter, res.t_exit), cols):
        assert got.ctypes.data == want.ctypes.data  # a view, not a copy
        assert np.array_equal(got, want)
    t_exit = res.t_exit
    del res, got, want
    gc.collect()
    assert freed == []  # one array still alive
    assert t_exit[-1] == 3.0
    del t_exit
    gc.collect()
    assert freed == [ctypes.addressof(r)]
