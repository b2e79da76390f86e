"""Thin ctypes binding of the libtdq C ABI (include/tdq.h).

Argument marshalling only: every step of the search runs in the CUDA library.
PyTorch is used for device memory and streams (device-resident inputs and the
caller's result buffers are torch CUDA tensors); host inputs are numpy arrays.
Names follow the C functions: build_index, search, search_device,
search_device_batched, get_stats, index_bins, last_error, version.

The library must be built (``paper_1405_7461_gb300.build.build()``); importing
this module without it raises, there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .workloads import COLUMNS, Segments

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdq.so")

TDQ_OK = 0
TDQ_ERR_INVALID = 1
TDQ_ERR_NOMEM = 2
TDQ_ERR_CUDA = 3
TDQ_ERR_TIMEOUT = 4
TDQ_ERR_OVERFLOW = 5
STATUS_NAMES = {0: "TDQ_OK", 1: "TDQ_ERR_INVALID", 2: "TDQ_ERR_NOMEM", 3: "TDQ_ERR_CUDA",
                4: "TDQ_ERR_TIMEOUT", 5: "TDQ_ERR_OVERFLOW"}
MODE_FP64 = 0
MODE_FP32_FILTER = 1
MODE_TC_FILTER = 2
FLAG_OTHER_TRAJECTORIES = 1  # TDQ_FLAG_OTHER_TRAJECTORIES
FLAG_UNORDERED_ONCE = 2  # TDQ_FLAG_UNORDERED_ONCE

c_dbl_p = ctypes.c_void_p


class tdq_segments(ctypes.Structure):
    _fields_ = [(c, ctypes.c_void_p) for c in COLUMNS] + [
        ("seg_id", ctypes.c_void_p), ("traj_id", ctypes.c_void_p), ("n", ctypes.c_uint64),
        ("on_device", ctypes.c_int)]


class tdq_index_params(ctypes.Structure):
    _fields_ = [("bin_count", ctypes.c_uint32)]


class tdq_search_params(ctypes.Structure):
    _fields_ = [("query_tile", ctypes.c_uint32), ("entry_chunk", ctypes.c_uint32), ("mode", ctypes.c_int),
                ("flags", ctypes.c_uint32)]


class tdq_results(ctypes.Structure):
    _fields_ = [("query_seg_id", ctypes.c_void_p), ("entry_seg_id", ctypes.c_void_p), ("t_enter", ctypes.c_void_p),
                ("t_exit", ctypes.c_void_p), ("count", ctypes.c_uint64)]


class tdq_result_buffer(ctypes.Structure):
    _fields_ = [("query_seg_id", ctypes.c_void_p), ("entry_seg_id", ctypes.c_void_p), ("t_enter", ctypes.c_void_p),
                ("t_exit", ctypes.c_void_p), ("capacity", ctypes.c_uint64)]


class tdq_stats(ctypes.Structure):
    _fields_ = [("query_segments", ctypes.c_uint64), ("interactions", ctypes.c_uint64),
                ("overlap_pairs", ctypes.c_uint64), ("fp64_pairs", ctypes.c_uint64), ("results", ctypes.c_uint64),
                ("work_items", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("pair_kernel_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("filter_survivors", ctypes.c_uint64), ("refine_ms", ctypes.c_double),
                ("mma_issued", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class tdq_plan_params(ctypes.Structure):
    _fields_ = [("max_query_segments", ctypes.c_uint64), ("result_capacity", ctypes.c_uint64),
                ("entry_chunk", ctypes.c_uint32), ("mode", ctypes.c_int), ("no_graph", ctypes.c_int),
                ("host_results", ctypes.c_int)]


class tdq_autotune_params(ctypes.Structure):
    _fields_ = [("bin_counts", ctypes.c_void_p), ("n_bin_counts", ctypes.c_int), ("entry_chunks", ctypes.c_void_p),
                ("n_entry_chunks", ctypes.c_int), ("batch_sizes", ctypes.c_void_p), ("n_batch_sizes", ctypes.c_int),
                ("mode", ctypes.c_int), ("repeats", ctypes.c_int), ("batch_tolerance", ctypes.c_double)]


class tdq_tuning(ctypes.Structure):
    _fields_ = [("bin_count", ctypes.c_uint32), ("entry_chunk", ctypes.c_uint32),
                ("batch_query_segments", ctypes.c_uint64), ("result_capacity", ctypes.c_uint64),
                ("ms_per_query_segment", ctypes.c_double), ("results_per_query_segment", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class tdq_server_params(ctypes.Structure):
    _fields_ = [("max_batch_query_segments", ctypes.c_uint64), ("memory_cap_bytes", ctypes.c_uint64),
                ("lanes", ctypes.c_int), ("mode", ctypes.c_int), ("entry_chunk", ctypes.c_uint32),
                ("results_per_query_segment", ctypes.c_double)]


class tdq_request_info(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("batch", ctypes.c_uint64), ("batch_query_segments", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class tdq_server_stats(ctypes.Structure):
    _fields_ = [("requests_submitted", ctypes.c_uint64), ("requests_completed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("failed_batches", ctypes.c_uint64),
                ("query_segments", ctypes.c_uint64), ("max_concurrent_batches", ctypes.c_uint64),
                ("peak_bytes_in_flight", ctypes.c_double), ("queued", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# Every symbol include/tdq.h declares, with (restype, argtypes).
P = ctypes.c_void_p
SIGNATURES = {
    "tdq_build_index": (ctypes.c_int, [P, P, P, P]),
    "tdq_index_free": (None, [P]),
    "tdq_index_size": (ctypes.c_uint64, [P]),
    "tdq_index_bins": (ctypes.c_int, [P, P, P, P, P, P, P, P, P]),
    "tdq_search": (ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P]),
    "tdq_self_join": (ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P]),
    "tdq_results_free": (None, [P]),
    "tdq_search_device": (ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P, P]),
    "tdq_search_device_batched": (ctypes.c_int, [P, P, P, P, P, P, P, P, P]),
    "tdq_search_device_noalloc": (ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P,
                                                 P]),
    "tdq_get_stats": (ctypes.c_int, [P, P]),
    "tdq_plan_create": (ctypes.c_int, [P, P, P]),
    "tdq_plan_free": (None, [P]),
    "tdq_plan_search": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "tdq_plan_results": (ctypes.c_int, [P, P, P]),
    "tdq_plan_get_stats": (ctypes.c_int, [P, P]),
    "tdq_plan_copy_results": (ctypes.c_int, [P, P, P, P, P, ctypes.c_uint64, ctypes.c_int, P]),
    "tdq_autotune": (ctypes.c_int, [P, P, P, P, P, P, P, P]),
    "tdq_server_create": (ctypes.c_int, [P, P, P]),
    "tdq_server_submit": (ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P]),
    "tdq_server_submit_many": (ctypes.c_int, [P, P, P, ctypes.c_uint64, P, P, P, P]),
    "tdq_server_drain": (ctypes.c_int, [P, ctypes.c_int64]),
    "tdq_server_wait": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_int64, P, P]),
    "tdq_server_get_stats": (ctypes.c_int, [P, P]),
    "tdq_server_free": (None, [P]),
    "tdq_last_error": (ctypes.c_char_p, []),
    "tdq_debug_fail_allocations": (None, [ctypes.c_int64]),
    "tdq_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libtdq.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libtdq.so not found at {path}: build it with paper_1405_7461_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class TdqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def debug_fail_allocations(after: int) -> None:
    """tdq_debug_fail_allocations: make the allocation `after` allocations
    from now fail once (after < 0: off)."""
    load().tdq_debug_fail_allocations(int(after))


def last_error() -> str:
    return load().tdq_last_error().decode()


def version() -> str:
    return load().tdq_version().decode()


def _check(st):
    if st != TDQ_OK:
        raise TdqError(st, last_error())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


# --------------------------------------------------------------------------
# Segment marshalling
# --------------------------------------------------------------------------

class HostSegments:
    """Host (numpy) columns of a segment set, kept alive for the call."""

    def __init__(self, seg: Segments):
        self.cols = [np.ascontiguousarray(getattr(seg, c), dtype=np.float64) for c in COLUMNS]
        self.seg_id = np.ascontiguousarray(seg.seg_id, dtype=np.int64)
        self.traj_id = np.ascontiguousarray(seg.traj_id, dtype=np.int64)
        self.n = len(self.cols[0])

    def struct(self) -> tdq_segments:
        s = tdq_segments()
        for c, a in zip(COLUMNS, self.cols):
            setattr(s, c, a.ctypes.data)
        s.seg_id = self.seg_id.ctypes.data
        s.traj_id = self.traj_id.ctypes.data
        s.n = self.n
        s.on_device = 0
        return s


class DeviceSegments:
    """Device (torch CUDA tensor) columns of a segment set."""

    def __init__(self, seg: Segments | None = None, device="cuda", tensors=None):
        import torch

        if tensors is not None:
            self.cols, self.seg_id, self.traj_id = tensors
        else:
            self.cols = [torch.from_numpy(np.ascontiguousarray(getattr(seg, c), np.float64)).to(device)
                         for c in COLUMNS]
            self.seg_id = torch.from_numpy(np.ascontiguousarray(seg.seg_id, np.int64)).to(device)
            self.traj_id = torch.from_numpy(np.ascontiguousarray(seg.traj_id, np.int64)).to(device)
        self.n = int(self.cols[0].shape[0])

    def struct(self) -> tdq_segments:
        # reused while the same tensor objects are attached
        key = (id(self.cols), tuple(id(c) for c in self.cols), id(self.seg_id), id(self.traj_id), self.n)
        cached = getattr(self, "_struct", None)
        if cached is not None and cached[0] == key:
            return cached[1]
        s = tdq_segments()
        for c, a in zip(COLUMNS, self.cols):
            if not (a.is_cuda and a.is_contiguous() and a.dtype == self._f64()):
                raise ValueError("tdq: device columns must be contiguous CUDA float64 tensors")
            setattr(s, c, a.data_ptr() if self.n else None)
        s.seg_id = self.seg_id.data_ptr() if self.n else None
        s.traj_id = self.traj_id.data_ptr() if self.n else None
        s.n = self.n
        s.on_device = 1
        self._struct = (key, s)
        return s

    @staticmethod
    def _f64():
        import torch

        return torch.float64

    @property
    def nbytes(self):
        return sum(c.numel() * 8 for c in self.cols) + 16 * self.n


def _segments(seg):
    if isinstance(seg, (HostSegments, DeviceSegments)):
        return seg
    if isinstance(seg, Segments):
        return HostSegments(seg)
    raise TypeError(f"expected Segments, HostSegments or DeviceSegments, got {type(seg)}")


def _params(query_tile=0, entry_chunk=0, mode=MODE_FP64, flags=0):
    p = tdq_search_params()
    p.query_tile = query_tile
    p.entry_chunk = entry_chunk
    p.mode = mode
    p.flags = flags
    return p


# --------------------------------------------------------------------------
# Index
# --------------------------------------------------------------------------

class Index:
    """Owner of a tdq_index handle."""

    def __init__(self, handle, n):
        self._h = handle
        self.n = n

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("index has been freed")
        return self._h

    def free(self):
        if self._h:
            load().tdq_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.free()


def build_index(entries, bin_count: int = 0, stream=None) -> Index:
    """tdq_build_index: temporal-bin index over the entry segments."""
    lib = load()
    seg = _segments(entries)
    s = seg.struct()
    prm = tdq_index_params(bin_count)
    h = ctypes.c_void_p()
    _check(lib.tdq_build_index(ctypes.byref(s), ctypes.byref(prm), _stream_ptr(stream), ctypes.byref(h)))
    return Index(h.value, seg.n)


def index_size(idx: Index) -> int:
    return int(load().tdq_index_size(idx.handle))


def index_bins(idx: Index, with_order: bool = False):
    """tdq_index_bins: the bin table (start, end, first, last) and bin width."""
    lib = load()
    m = ctypes.c_uint32()
    width = ctypes.c_double()
    tmin = ctypes.c_double()
    _check(lib.tdq_index_bins(idx.handle, ctypes.byref(m), None, None, None, None, None, None, None))
    mm = m.value
    bs = np.empty(mm, np.float64)
    be = np.empty(mm, np.float64)
    bf = np.empty(mm, np.int64)
    bl = np.empty(mm, np.int64)
    order = np.empty(idx.n, np.int64) if with_order else None
    _check(lib.tdq_index_bins(idx.handle, ctypes.byref(m), ctypes.byref(width), ctypes.byref(tmin), bs.ctypes.data,
                              be.ctypes.data, bf.ctypes.data, bl.ctypes.data,
                              order.ctypes.data if with_order and idx.n else None))
    out = {"m": mm, "width": width.value, "t_min": tmin.value, "start": bs, "end": be, "first": bf, "last": bl}
    if with_order:
        out["order"] = order
    return out


@dataclass
class Results:
    query_seg_id: np.ndarray
    entry_seg_id: np.ndarray
    t_enter: np.ndarray
    t_exit: np.ndarray

    def __len__(self):
        return len(self.query_seg_id)


def search(idx: Index, queries, d: float, t0: float = -np.inf, t1: float = np.inf, stream=None,
           **params) -> Results:
    """tdq_search: results copied to host memory (the library retries on overflow)."""
    return _host_results("tdq_search", idx, queries, d, t0, t1, stream, params)


def self_join(idx: Index, entries, d: float, t0: float = -np.inf, t1: float = np.inf, stream=None,
              **params) -> Results:
    """tdq_self_join: every pair of segments of different trajectories of
    the indexed set (`entries`, the segments the index was built from) within
    d, each unordered pair once (query_seg_id < entry_seg_id)."""
    return _host_results("tdq_self_join", idx, entries, d, t0, t1, stream, params)


def _host_results(fn, idx, queries, d, t0, t1, stream, params) -> Results:
    lib = load()
    q = _segments(queries)
    s = q.struct()
    prm = _params(**params)
    out = ctypes.POINTER(tdq_results)()
    _check(getattr(lib, fn)(idx.handle, ctypes.byref(s), float(d), float(t0), float(t1), ctypes.byref(prm),
                            _stream_ptr(stream), ctypes.byref(out)))
    return _take_results(out)


class _LibResults:
    """Owner of a library-allocated tdq_results: the numpy arrays handed out
    are views of its columns (no copy); it is released with tdq_results_free
    when the last of them is gone."""

    def __init__(self, ptr):
        self._ptr = ptr

    def __del__(self):
        lib = _lib  # None once the module is torn down at exit
        if self._ptr is not None and lib is not None:
            lib.tdq_results_free(self._ptr)
            self._ptr = None


class DeviceResultBuffer:
    """Caller-owned device result buffer (torch tensors)."""

    def __init__(self, capacity: int, device="cuda"):
        import torch

        self.capacity = int(capacity)
        self.query_seg_id = torch.empty(max(1, capacity), dtype=torch.int64, device=device)
        self.entry_seg_id = torch.empty(max(1, capacity), dtype=torch.int64, device=device)
        self.t_enter = torch.empty(max(1, capacity), dtype=torch.float64, device=device)
        self.t_exit = torch.empty(max(1, capacity), dtype=torch.float64, device=device)

    def struct(self) -> tdq_result_buffer:
        b = tdq_result_buffer()
        b.query_seg_id = self.query_seg_id.data_ptr()
        b.entry_seg_id = self.entry_seg_id.data_ptr()
        b.t_enter = self.t_enter.data_ptr()
        b.t_exit = self.t_exit.data_ptr()
        b.capacity = self.capacity
        return b

    def to_host(self, count: int) -> Results:
        count = min(count, self.capacity)
        return Results(self.query_seg_id[:count].cpu().numpy(), self.entry_seg_id[:count].cpu().numpy(),
                       self.t_enter[:count].cpu().numpy(), self.t_exit[:count].cpu().numpy())


def search_device(idx: Index, queries: DeviceSegments, d: float, t0: float, t1: float,
                  out: DeviceResultBuffer, stream=None, allow_overflow=False, **params) -> int:
    """tdq_search_device: returns the result count (raises on overflow unless allowed)."""
    lib = load()
    s = queries.struct()
    prm = _params(**params)
    b = out.struct()
    cnt = ctypes.c_uint64()
    st = lib.tdq_search_device(idx.handle, ctypes.byref(s), float(d), float(t0), float(t1), ctypes.byref(prm),
                               _stream_ptr(stream), ctypes.byref(b), ctypes.byref(cnt))
    if st == TDQ_ERR_OVERFLOW and allow_overflow:
        return int(cnt.value)
    _check(st)
    return int(cnt.value)


def search_device_batched(idx: Index, queries: DeviceSegments, d_per_query, t0_per_query, t1_per_query,
                          out: DeviceResultBuffer, stream=None, allow_overflow=False, **params) -> int:
    """tdq_search_device_batched: per-query-segment d and window (torch CUDA float64 tensors)."""
    lib = load()
    s = queries.struct()
    prm = _params(**params)
    b = out.struct()
    cnt = ctypes.c_uint64()
    for t in (d_per_query, t0_per_query, t1_per_query):
        assert t.is_cuda and t.dtype.itemsize == 8 and t.is_contiguous()
    st = lib.tdq_search_device_batched(idx.handle, ctypes.byref(s), d_per_query.data_ptr(), t0_per_query.data_ptr(),
                                       t1_per_query.data_ptr(), ctypes.byref(prm), _stream_ptr(stream),
                                       ctypes.byref(b), ctypes.byref(cnt))
    if st == TDQ_ERR_OVERFLOW and allow_overflow:
        return int(cnt.value)
    _check(st)
    return int(cnt.value)


NOALLOC_MAX_QUERIES = 8192


def search_device_noalloc(idx: Index, queries: DeviceSegments, d: float, t0: float, t1: float,
                          out: DeviceResultBuffer, stream=None, allow_overflow=False, **params) -> int:
    """tdq_search_device_noalloc: same as search_device, but the library
    allocates nothing (scratch in a fixed device array; at most
    NOALLOC_MAX_QUERIES query segments per call; calls must not overlap)."""
    lib = load()
    s = queries.struct()
    prm = _params(**params)
    b = out.struct()
    cnt = ctypes.c_uint64()
    st = lib.tdq_search_device_noalloc(idx.handle, ctypes.byref(s), float(d), float(t0), float(t1),
                                       ctypes.byref(prm), _stream_ptr(stream), ctypes.byref(b), ctypes.byref(cnt))
    if st == TDQ_ERR_OVERFLOW and allow_overflow:
        return int(cnt.value)
    _check(st)
    return int(cnt.value)


def get_stats(idx: Index) -> dict:
    st = tdq_stats()
    _check(load().tdq_get_stats(idx.handle, ctypes.byref(st)))
    return st.as_dict()


# --------------------------------------------------------------------------
# Batched plans (CUDA graph) and the autotuner
# --------------------------------------------------------------------------

def _per_query_ptrs(queries, d, t0, t1):
    """Pointers of the per-query d / t0 / t1 arrays, in the queries' memory."""
    if isinstance(queries, DeviceSegments):
        import torch

        dev = queries.cols[0].device
        if all(getattr(a, "is_cuda", False) and a.dtype == torch.float64 and a.device == dev and a.is_contiguous()
               for a in (d, t0, t1)):
            return None, [a.data_ptr() for a in (d, t0, t1)]  # already in place: no copies
        keep = [torch.as_tensor(np.asarray(a, np.float64) if not hasattr(a, "is_cuda") else a,
                                dtype=torch.float64).to(dev).contiguous() for a in (d, t0, t1)]
        return keep, [k.data_ptr() for k in keep]
    keep = [np.ascontiguousarray(a, np.float64) for a in (d, t0, t1)]
    return keep, [k.ctypes.data for k in keep]


class Plan:
    """Owner of a tdq_plan: batches of query segments with their own d and
    window, each batch one CUDA graph launch."""

    def __init__(self, idx: Index, max_query_segments: int, mode=MODE_FP64, entry_chunk=0, result_capacity=0,
                 use_graph=True, host_results=False):
        self.idx = idx
        self.host_results = bool(host_results)
        prm = tdq_plan_params(int(max_query_segments), int(result_capacity), int(entry_chunk), int(mode),
                              0 if use_graph else 1, 1 if host_results else 0)
        h = ctypes.c_void_p()
        _check(load().tdq_plan_create(idx.handle, ctypes.byref(prm), ctypes.byref(h)))
        self._h = h.value

    def free(self):
        if self._h:
            load().tdq_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.free()

    def search(self, queries, d, t0, t1, stream=None) -> int:
        """tdq_plan_search: d, t0, t1 per query segment; returns the result count."""
        q = _segments(queries)
        s = q.struct()
        keep, ptrs = _per_query_ptrs(q, d, t0, t1)
        cnt = ctypes.c_uint64()
        _check(load().tdq_plan_search(self._h, ctypes.byref(s), *ptrs, _stream_ptr(stream), ctypes.byref(cnt)))
        del keep
        return int(cnt.value)

    def results(self, out=None, view=False) -> Results:
        """tdq_plan_copy_results: the last batch's results, copied to host --
        into new arrays, or into `out` = (query_seg_id, entry_seg_id,
        t_enter, t_exit), caller arrays (e.g. pinned memory) large enough for
        the count, returned as views of their first entries.  view=True (a
        plan with host_results): arrays over the plan's own page-locked
        result buffer, where the kernels wrote them -- no copy; valid until
        the next search on the plan or its release."""
        buf = tdq_result_buffer()
        cnt = ctypes.c_uint64()
        _check(load().tdq_plan_results(self._h, ctypes.byref(buf), ctypes.byref(cnt)))
        n = int(cnt.value)
        if view:
            if not self.host_results:
                raise ValueError("tdq: results(view=True) needs a plan created with host_results=True")

            def arr(p, dt):
                if n == 0:
                    return np.empty(0, dt)
                return np.frombuffer((ctypes.c_char * (n * 8)).from_address(p), dtype=dt)

            return Results(arr(buf.query_seg_id, np.int64), arr(buf.entry_seg_id, np.int64),
                           arr(buf.t_enter, np.float64), arr(buf.t_exit, np.float64))
        if out is not None:
            if any(len(a) < n or not a.flags["C_CONTIGUOUS"] for a in out):
                raise ValueError("tdq: result arrays too small or not contiguous")
            if out[0].dtype != np.int64 or out[1].dtype != np.int64 or out[2].dtype != np.float64 \
                    or out[3].dtype != np.float64:
                raise ValueError("tdq: result arrays must be int64, int64, float64, float64")
            qi, ei, tin, tout = (a[:n] for a in out)
        else:
            qi = np.empty(n, np.int64)
            ei = np.empty(n, np.int64)
            tin = np.empty(n, np.float64)
            tout = np.empty(n, np.float64)
        if n:
            _check(load().tdq_plan_copy_results(self._h, qi.ctypes.data, ei.ctypes.data, tin.ctypes.data,
                                                tout.ctypes.data, n, 0, None))
        return Results(qi, ei, tin, tout)

    def stats(self) -> dict:
        st = tdq_stats()
        _check(load().tdq_plan_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()


def autotune(entries, sample, d, t0, t1, mode=MODE_FP64, bin_counts=None, entry_chunks=None, batch_sizes=None,
             repeats=3, batch_tolerance=0.05, stream=None) -> dict:
    """tdq_autotune: measured bin count, entry chunk and batch size."""
    e = _segments(entries)
    q = _segments(sample)
    es, qs = e.struct(), q.struct()
    keep, ptrs = _per_query_ptrs(q, d, t0, t1)
    ap = tdq_autotune_params()
    arrs = []
    if bin_counts is not None:
        a = np.ascontiguousarray(bin_counts, np.uint32)
        arrs.append(a)
        ap.bin_counts, ap.n_bin_counts = a.ctypes.data, len(a)
    if entry_chunks is not None:
        a = np.ascontiguousarray(entry_chunks, np.uint32)
        arrs.append(a)
        ap.entry_chunks, ap.n_entry_chunks = a.ctypes.data, len(a)
    if batch_sizes is not None:
        a = np.ascontiguousarray(batch_sizes, np.uint64)
        arrs.append(a)
        ap.batch_sizes, ap.n_batch_sizes = a.ctypes.data, len(a)
    ap.mode = mode
    ap.repeats = repeats
    ap.batch_tolerance = batch_tolerance
    out = tdq_tuning()
    _check(load().tdq_autotune(ctypes.byref(es), ctypes.byref(qs), *ptrs, ctypes.byref(ap), _stream_ptr(stream),
                               ctypes.byref(out)))
    del keep, arrs
    return out.as_dict()


# --------------------------------------------------------------------------
# Serving loop
# --------------------------------------------------------------------------

def _take_results(ptr) -> Results:
    """Results over a library-allocated tdq_results (no copy): the arrays are
    views of its columns, released with tdq_results_free when the last of
    them is gone."""
    owner = _LibResults(ptr)
    r = ptr.contents
    n = int(r.count)

    def arr(p, dt):
        if n == 0:
            return np.empty(0, dt)
        buf = (ctypes.c_char * (n * 8)).from_address(p)
        buf._owner = owner  # the library's arrays live as long as any view of them
        return np.frombuffer(buf, dtype=dt)

    return Results(arr(r.query_seg_id, np.int64), arr(r.entry_seg_id, np.int64), arr(r.t_enter, np.float64),
                   arr(r.t_exit, np.float64))


class Server:
    """Owner of a tdq_server: continuous batching over a resident index."""

    def __init__(self, idx: Index, max_batch_query_segments=65536, memory_cap_bytes=16 << 30, lanes=2,
                 mode=MODE_FP32_FILTER, entry_chunk=0, results_per_query_segment=0.0):
        self.idx = idx
        prm = tdq_server_params(int(max_batch_query_segments), int(memory_cap_bytes), int(lanes), int(mode),
                                int(entry_chunk), float(results_per_query_segment))
        h = ctypes.c_void_p()
        _check(load().tdq_server_create(idx.handle, ctypes.byref(prm), ctypes.byref(h)))
        self._h = h.value

    def submit(self, query: Segments, d: float, t0: float, t1: float) -> int:
        q = HostSegments(query)
        s = q.struct()
        t = ctypes.c_uint64()
        _check(load().tdq_server_submit(self._h, ctypes.byref(s), float(d), float(t0), float(t1), ctypes.byref(t)))
        return int(t.value)

    def submit_many(self, queries, d, t0, t1) -> list:
        """tdq_server_submit_many: queue several requests in one call;
        queries is a list of Segments (one per request), d / t0 / t1 one
        value per request.  Returns their tickets."""
        k = len(queries)
        if k == 0:
            return []
        cat = Segments.concat(list(queries))
        offs = np.zeros(k + 1, np.uint64)
        offs[1:] = np.cumsum([len(q) for q in queries])
        dd, a0, a1 = (np.ascontiguousarray(np.asarray(x, np.float64)) for x in (d, t0, t1))
        assert len(dd) == len(a0) == len(a1) == k
        tickets = np.zeros(k, np.uint64)
        q = HostSegments(cat)
        s = q.struct()
        _check(load().tdq_server_submit_many(self._h, ctypes.byref(s), offs.ctypes.data, k, dd.ctypes.data,
                                             a0.ctypes.data, a1.ctypes.data, tickets.ctypes.data))
        return [int(t) for t in tickets]

    def drain(self, timeout_ms: int = -1) -> None:
        """tdq_server_drain: wait until every submitted request has been searched."""
        _check(load().tdq_server_drain(self._h, int(timeout_ms)))

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Results and timing info of a request (raises TdqError with
        TDQ_ERR_TIMEOUT if it is not done within timeout_ms)."""
        out = ctypes.POINTER(tdq_results)()
        info = tdq_request_info()
        _check(load().tdq_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(out), ctypes.byref(info)))
        return _take_results(out), info.as_dict()

    def stats(self) -> dict:
        st = tdq_server_stats()
        _check(load().tdq_server_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def free(self):
        if self._h:
            load().tdq_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.free()
