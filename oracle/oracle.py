"""Python access to the CPU FP64 oracle (``tdq_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports, links or calls anything here, and this module never touches it.

Segments are passed as the eight columns of the paper's data model (Sec. 3):
start point (x, y, z, t) and end point (x, y, z, t), as float64 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdq_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
COLUMNS = ("xs", "ys", "zs", "ts", "xe", "ye", "ze", "te")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def build_mutant(k: int, out_dir: str) -> str:
    """Compile the oracle with deliberate mistake number k planted (the
    test-suite checks that its pins catch every one)."""
    path = os.path.join(out_dir, "liboracle_mutant%d.so" % k)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                           "-DORACLE_MUTANT=%d" % k, "-o", path, _SRC, "-lm"])
    return path


def use_library(path):
    """Make the module call the oracle library at `path` (None: the normal
    build).  Returns the previous library handle."""
    global _lib
    prev = _lib
    _lib = _configure(ctypes.CDLL(path)) if path else None
    return prev


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    if True:
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        dbl = ctypes.c_double
        lib.oracle_pair.restype = ctypes.c_int
        lib.oracle_pair.argtypes = [P, P, dbl, dbl, dbl, P, P, P]
        for name in ("oracle_search_bruteforce", "oracle_search_sweep"):
            f = getattr(lib, name)
            f.restype = P
            f.argtypes = [P, i64, P, i64, dbl, dbl, dbl, ctypes.c_int]
        lib.oracle_search_sweep_per_query.restype = P
        lib.oracle_search_sweep_per_query.argtypes = [P, i64, P, i64, P, P, P, ctypes.c_int]
        lib.oracle_self_join.restype = P
        lib.oracle_self_join.argtypes = [P, i64, P, P, dbl, dbl, dbl, ctypes.c_int]
        lib.oracle_result_count.restype = i64
        lib.oracle_result_count.argtypes = [P]
        lib.oracle_result_overlap_pairs.restype = i64
        lib.oracle_result_overlap_pairs.argtypes = [P]
        lib.oracle_result_visited_pairs.restype = i64
        lib.oracle_result_visited_pairs.argtypes = [P]
        lib.oracle_result_copy.restype = None
        lib.oracle_result_copy.argtypes = [P, P, P, P, P, P]
        lib.oracle_result_free.restype = None
        lib.oracle_result_free.argtypes = [P]
        lib.oracle_default_threads.restype = ctypes.c_int
        lib.oracle_bin_table.restype = dbl
        lib.oracle_bin_table.argtypes = [P, P, i64, i64, P, P, P, P, P]
        lib.oracle_batch_interactions.restype = i64
        lib.oracle_batch_interactions.argtypes = [P, P, P, P, i64, P, P, P, i64]
    return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _columns(seg) -> tuple[list[np.ndarray], ctypes.Array]:
    cols = [np.ascontiguousarray(seg[c], dtype=np.float64) for c in COLUMNS]
    arr = (ctypes.c_void_p * 8)(*[_ptr(c) for c in cols])
    return cols, arr


@dataclass
class OracleResult:
    """Reported pairs, as indices into the query and entry inputs."""

    query_index: np.ndarray
    entry_index: np.ndarray
    t_enter: np.ndarray
    t_exit: np.ndarray
    dmin: np.ndarray
    overlap_pairs: int
    visited_pairs: int

    def sorted(self) -> "OracleResult":
        o = np.lexsort((self.entry_index, self.query_index))
        return OracleResult(self.query_index[o], self.entry_index[o], self.t_enter[o], self.t_exit[o],
                            self.dmin[o], self.overlap_pairs, self.visited_pairs)


def default_threads() -> int:
    return int(_load().oracle_default_threads())


def _collect(lib, h):
    if not h:
        raise MemoryError("oracle search failed to allocate")
    try:
        cnt = lib.oracle_result_count(h)
        qi = np.empty(cnt, np.int64)
        ei = np.empty(cnt, np.int64)
        tin = np.empty(cnt, np.float64)
        tout = np.empty(cnt, np.float64)
        dm = np.empty(cnt, np.float64)
        if cnt:
            lib.oracle_result_copy(h, _ptr(qi), _ptr(ei), _ptr(tin), _ptr(tout), _ptr(dm))
        res = OracleResult(qi, ei, tin, tout, dm, int(lib.oracle_result_overlap_pairs(h)),
                           int(lib.oracle_result_visited_pairs(h)))
    finally:
        lib.oracle_result_free(h)
    return res.sorted()


def _search(fn_name, entries, queries, d, t0, t1, threads):
    lib = _load()
    ecols, earr = _columns(entries)
    qcols, qarr = _columns(queries)
    n = len(ecols[0])
    nq = len(qcols[0])
    h = getattr(lib, fn_name)(ctypes.cast(earr, ctypes.c_void_p), n, ctypes.cast(qarr, ctypes.c_void_p),
                              nq, float(d), float(t0), float(t1), int(threads))
    res = _collect(lib, h)
    del ecols, qcols
    return res


def search_bruteforce(entries, queries, d, t0=-np.inf, t1=np.inf, threads=0) -> OracleResult:
    """Every query segment against every entry segment."""
    return _search("oracle_search_bruteforce", entries, queries, d, t0, t1, threads)


def search_sweep(entries, queries, d, t0=-np.inf, t1=np.inf, threads=0) -> OracleResult:
    """Same result as :func:`search_bruteforce`, visiting only pairs whose starts can overlap."""
    return _search("oracle_search_sweep", entries, queries, d, t0, t1, threads)


def search_sweep_per_query(entries, queries, d, t0, t1, threads=0) -> OracleResult:
    """The time sweep with query segment i searched at its own threshold
    d[i] over its own window [t0[i], t1[i]] (arrays, one value per query
    segment)."""
    lib = _load()
    ecols, earr = _columns(entries)
    qcols, qarr = _columns(queries)
    nq = len(qcols[0])
    dd, w0, w1 = (np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), (nq,))) for a in (d, t0, t1))
    h = lib.oracle_search_sweep_per_query(ctypes.cast(earr, ctypes.c_void_p), len(ecols[0]),
                                          ctypes.cast(qarr, ctypes.c_void_p), nq, _ptr(dd), _ptr(w0), _ptr(w1),
                                          int(threads))
    res = _collect(lib, h)
    del ecols, qcols, dd, w0, w1
    return res


def self_join(entries, d, t0=-np.inf, t1=np.inf, threads=0) -> OracleResult:
    """Query (ii) of Sec. 2.1 with the database as the query set: every
    segment against the segments of every other trajectory, each unordered
    pair once (query index = the segment with the smaller seg_id).  The
    overlap count covers all pairs, the left-out ones included."""
    lib = _load()
    ecols, earr = _columns(entries)
    traj = np.ascontiguousarray(entries.traj_id, np.int64)
    seg = np.ascontiguousarray(entries.seg_id, np.int64)
    h = lib.oracle_self_join(ctypes.cast(earr, ctypes.c_void_p), len(ecols[0]), _ptr(traj), _ptr(seg), float(d),
                             float(t0), float(t1), int(threads))
    res = _collect(lib, h)
    del ecols, traj, seg
    return res


def pair(e8, q8, d, t0=-np.inf, t1=np.inf):
    """One pair.  Returns (status, t_enter, t_exit, dmin): status -1 no common
    span, 0 common span but never within d, 1 within d over [t_enter, t_exit]."""
    lib = _load()
    e = np.ascontiguousarray(e8, dtype=np.float64)
    q = np.ascontiguousarray(q8, dtype=np.float64)
    assert e.shape == (8,) and q.shape == (8,)
    tin = ctypes.c_double(np.nan)
    tout = ctypes.c_double(np.nan)
    dm = ctypes.c_double(np.nan)
    st = lib.oracle_pair(_ptr(e), _ptr(q), float(d), float(t0), float(t1), ctypes.byref(tin),
                         ctypes.byref(tout), ctypes.byref(dm))
    return int(st), tin.value, tout.value, dm.value


def pair_dmin(entries, ei, queries, qi, t0=-np.inf, t1=np.inf):
    """Distance of closest approach of entry ei and query qi inside their common
    span (NaN when they share no span of positive length)."""
    e8 = np.array([entries[c][ei] for c in COLUMNS], np.float64)
    q8 = np.array([queries[c][qi] for c in COLUMNS], np.float64)
    st, _, _, dm = pair(e8, q8, 0.0, t0, t1)
    return np.nan if st < 0 else dm


def bin_table(ts, te, m):
    """The temporal-bin index of Sec. 4 (Fig. 1).  Returns a dict with the
    sorted order, the bin width b and per-bin start (smallest t_start), end
    (largest t_end), first and last sorted positions (-1 for empty bins)."""
    lib = _load()
    ts = np.ascontiguousarray(ts, np.float64)
    te = np.ascontiguousarray(te, np.float64)
    n = len(ts)
    order = np.empty(n, np.int64)
    bs = np.empty(m, np.float64)
    be = np.empty(m, np.float64)
    bf = np.empty(m, np.int64)
    bl = np.empty(m, np.int64)
    b = lib.oracle_bin_table(_ptr(ts), _ptr(te), n, m, _ptr(order), _ptr(bs), _ptr(be), _ptr(bf), _ptr(bl))
    return {"order": order, "width": b, "start": bs, "end": be, "first": bf, "last": bl}


def batch_interactions(bin_lo, bin_end, bin_first, bin_last, counts, bts, bte) -> int:
    """Interactions of a query batching over a bin table (Sec. 4, Fig. 2)."""
    lib = _load()
    bin_lo = np.ascontiguousarray(bin_lo, np.float64)
    bin_end = np.ascontiguousarray(bin_end, np.float64)
    bin_first = np.ascontiguousarray(bin_first, np.int64)
    bin_last = np.ascontiguousarray(bin_last, np.int64)
    counts = np.ascontiguousarray(counts, np.int64)
    bts = np.ascontiguousarray(bts, np.float64)
    bte = np.ascontiguousarray(bte, np.float64)
    return int(lib.oracle_batch_interactions(_ptr(bin_lo), _ptr(bin_end), _ptr(bin_first), _ptr(bin_last),
                                             len(bin_lo), _ptr(counts), _ptr(bts), _ptr(bte), len(counts)))
