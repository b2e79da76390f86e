"""Seeded synthetic trajectory workloads.

These generators stand in for the paper's datasets (Galaxy and the RandWalk
family, Sec. 7.1, Table 1), which are not available here.  They only draw
trajectories; none of the search arithmetic lives in this module, so both the
CUDA path and the CPU oracle can be fed from it.

A trajectory is a polyline through points sampled at unit time steps; each pair
of consecutive points is one segment (Sec. 3: start point, end point, segment
id, trajectory id).  T points give T-1 segments.  Segment ids are global
running indices, increasing along each trajectory.

Workloads (sizes as named in their docstrings):
  tiny_random_walk   200 walks x 100 points, uniform steps, 20 queries, d=5
  scale_random_walk  10,000 walks, 100-400 points, Normal(0,1) steps, 100 queries
  galaxy_disk        50,000 stars on perturbed circular orbits, 200 points, 500 queries
  batching_walks     20,000 walks x 300 points, exponential step lengths, 5,000
                     fresh query walks with their own d and window
  serving_walks      40,000 walks x 500 points resident, Poisson query arrivals
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 14057461
COLUMNS = ("xs", "ys", "zs", "ts", "xe", "ye", "ze", "te")


@dataclass
class Segments:
    """Structure-of-arrays segment set: start (xs,ys,zs,ts), end (xe,ye,ze,te)."""

    xs: np.ndarray
    ys: np.ndarray
    zs: np.ndarray
    ts: np.ndarray
    xe: np.ndarray
    ye: np.ndarray
    ze: np.ndarray
    te: np.ndarray
    seg_id: np.ndarray
    traj_id: np.ndarray

    def __len__(self) -> int:
        return int(self.ts.shape[0])

    def __getitem__(self, name):
        return getattr(self, name)

    def take(self, idx) -> "Segments":
        idx = np.asarray(idx)
        return Segments(*[getattr(self, c)[idx] for c in COLUMNS], self.seg_id[idx], self.traj_id[idx])

    def row(self, i) -> np.ndarray:
        return np.array([getattr(self, c)[i] for c in COLUMNS], np.float64)

    @staticmethod
    def concat(parts) -> "Segments":
        return Segments(*[np.concatenate([getattr(p, c) for p in parts]) for c in COLUMNS],
                        np.concatenate([p.seg_id for p in parts]), np.concatenate([p.traj_id for p in parts]))

    @staticmethod
    def from_columns(cols, seg_id=None, traj_id=None) -> "Segments":
        n = len(cols[0])
        sid = np.arange(n, dtype=np.int64) if seg_id is None else np.asarray(seg_id, np.int64)
        tid = np.zeros(n, np.int64) if traj_id is None else np.asarray(traj_id, np.int64)
        return Segments(*[np.ascontiguousarray(c, dtype=np.float64) for c in cols], sid, tid)

    @property
    def nbytes(self) -> int:
        return sum(getattr(self, c).nbytes for c in COLUMNS) + self.seg_id.nbytes + self.traj_id.nbytes


@dataclass
class Workload:
    """Entries, queries and the search parameters of one synthetic workload."""

    name: str
    entries: Segments
    queries: Segments
    d_values: tuple
    window: tuple
    # per-query-segment threshold and window, for workloads where each query
    # trajectory carries its own (None otherwise)
    q_d: np.ndarray | None = None
    q_t0: np.ndarray | None = None
    q_t1: np.ndarray | None = None
    n_query_traj: int = 0
    meta: dict = field(default_factory=dict)


def polylines_to_segments(points, times, counts, traj_ids, first_seg_id=0) -> Segments:
    """Points (P,3) and times (P,) of consecutive trajectories with counts[k]
    points each -> the segments between consecutive points of each trajectory."""
    counts = np.asarray(counts, np.int64)
    P = int(counts.sum())
    assert points.shape == (P, 3) and times.shape == (P,)
    last = np.cumsum(counts) - 1  # index of the last point of each trajectory
    keep = np.ones(P, bool)
    keep[last] = False
    s = np.nonzero(keep)[0]
    e = s + 1
    tid = np.repeat(np.asarray(traj_ids, np.int64), counts - 1)
    nseg = len(s)
    return Segments(
        np.ascontiguousarray(points[s, 0]), np.ascontiguousarray(points[s, 1]),
        np.ascontiguousarray(points[s, 2]), np.ascontiguousarray(times[s]),
        np.ascontiguousarray(points[e, 0]), np.ascontiguousarray(points[e, 1]),
        np.ascontiguousarray(points[e, 2]), np.ascontiguousarray(times[e]),
        np.arange(first_seg_id, first_seg_id + nseg, dtype=np.int64), tid)


def _walk_points(starts, counts, steps):
    """Cumulative walk: point 0 of trajectory k is starts[k]; each next point
    adds the next row of steps.  steps has one row per point (the row of a
    trajectory's first point is ignored)."""
    counts = np.asarray(counts, np.int64)
    P = int(counts.sum())
    first = np.concatenate([[0], np.cumsum(counts)[:-1]])
    steps = steps.copy()
    steps[first] = 0.0
    cs = np.cumsum(steps, axis=0)
    traj_of_point = np.repeat(np.arange(len(counts)), counts)
    pts = cs - cs[first][traj_of_point] + starts[traj_of_point]
    assert pts.shape == (P, 3)
    return pts


def _unit_times(t_start, counts):
    counts = np.asarray(counts, np.int64)
    first = np.concatenate([[0], np.cumsum(counts)[:-1]])
    traj_of_point = np.repeat(np.arange(len(counts)), counts)
    k = np.arange(int(counts.sum())) - first[traj_of_point]
    return np.asarray(t_start, np.float64)[traj_of_point] + k.astype(np.float64)


def _queries_from_set(entries: Segments, rng, n_traj, n_queries):
    chosen = np.sort(rng.choice(n_traj, size=n_queries, replace=False))
    mask = np.isin(entries.traj_id, chosen)
    return entries.take(np.nonzero(mask)[0])


def tiny_random_walk(seed=DEFAULT_SEED, n_traj=200, n_points=100, n_queries=20) -> Workload:
    """200 walks x 100 points at t=0..99, start uniform in [0,100]^3, steps
    uniform in [-1,1]^3 (19,800 segments); 20 query trajectories taken from the
    set; d=5; window [0,99]."""
    rng = np.random.default_rng(seed)
    counts = np.full(n_traj, n_points, np.int64)
    starts = rng.uniform(0.0, 100.0, size=(n_traj, 3))
    steps = rng.uniform(-1.0, 1.0, size=(int(counts.sum()), 3))
    pts = _walk_points(starts, counts, steps)
    times = _unit_times(np.zeros(n_traj), counts)
    ent = polylines_to_segments(pts, times, counts, np.arange(n_traj))
    qry = _queries_from_set(ent, rng, n_traj, n_queries)
    return Workload("tiny_random_walk", ent, qry, (5.0,), (0.0, float(n_points - 1)),
                    n_query_traj=n_queries)


def scale_random_walk(seed=DEFAULT_SEED, n_traj=10_000, n_queries=100, min_points=100,
                      max_points=400, t_start_max=200.0) -> Workload:
    """10,000 walks, start time uniform in [0,200] (continuous), length uniform
    in 100..400 points, steps Normal(0,1) per axis, start uniform in
    [0,1000]^3; 100 query trajectories from the set; d in {1,5,15}; window =
    the full extent."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(min_points, max_points + 1, size=n_traj).astype(np.int64)
    t0 = rng.uniform(0.0, t_start_max, size=n_traj)
    starts = rng.uniform(0.0, 1000.0, size=(n_traj, 3))
    steps = rng.standard_normal(size=(int(counts.sum()), 3))
    pts = _walk_points(starts, counts, steps)
    times = _unit_times(t0, counts)
    ent = polylines_to_segments(pts, times, counts, np.arange(n_traj))
    qry = _queries_from_set(ent, rng, n_traj, n_queries)
    window = (float(ent.ts.min()), float(ent.te.max()))
    return Workload("scale_random_walk", ent, qry, (1.0, 5.0, 15.0), window, n_query_traj=n_queries)


KMS_TO_KPC_PER_MYR = 1.0227e-3


def galaxy_disk(seed=DEFAULT_SEED, n_stars=50_000, n_points=200, n_queries=500) -> Workload:
    """Disk-galaxy-shaped orbits (units kpc and Myr, dt = 1 Myr): radius
    exponential with scale length 3 truncated to [0.5,15], circular speed
    220 km/s with 10% Gaussian dispersion, random phase, vertical oscillation
    of amplitude Normal(0,0.3) kpc and period 85 Myr; 200 points per star
    (199 segments, 9.95 M for 50,000 stars); all start at t=0; 500 queries
    from the set; d in {0.01, 0.1, 1}."""
    rng = np.random.default_rng(seed)
    R = rng.exponential(3.0, size=n_stars)
    bad = (R < 0.5) | (R > 15.0)
    while bad.any():
        R[bad] = rng.exponential(3.0, size=int(bad.sum()))
        bad = (R < 0.5) | (R > 15.0)
    v = 220.0 * (1.0 + 0.1 * rng.standard_normal(n_stars)) * KMS_TO_KPC_PER_MYR
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n_stars)
    zamp = rng.normal(0.0, 0.3, size=n_stars)
    zph = rng.uniform(0.0, 2.0 * np.pi, size=n_stars)
    omega = v / R
    nu = 2.0 * np.pi / 85.0
    t = np.arange(n_points, dtype=np.float64)
    ang = phase[:, None] + omega[:, None] * t[None, :]
    pts = np.empty((n_stars * n_points, 3))
    pts[:, 0] = (R[:, None] * np.cos(ang)).ravel()
    pts[:, 1] = (R[:, None] * np.sin(ang)).ravel()
    pts[:, 2] = (zamp[:, None] * np.sin(nu * t[None, :] + zph[:, None])).ravel()
    counts = np.full(n_stars, n_points, np.int64)
    times = np.tile(t, n_stars)
    ent = polylines_to_segments(pts, times, counts, np.arange(n_stars))
    qry = _queries_from_set(ent, rng, n_stars, n_queries)
    return Workload("galaxy_disk", ent, qry, (0.01, 0.1, 1.0), (0.0, float(n_points - 1)),
                    n_query_traj=n_queries)


def _exp_isotropic_steps(rng, n):
    u = rng.standard_normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return u * rng.exponential(1.0, size=(n, 1))


def batching_walks(seed=DEFAULT_SEED, n_traj=20_000, n_points=300, n_queries=5_000, box=1000.0) -> Workload:
    """Entry database: 20,000 walks x 300 points (t=0..299), isotropic step
    direction with exponential length (mean 1), start uniform in [0,1000]^3
    (5.98 M segments).  5,000 fresh query walks: length lognormal(ln 63.2,
    0.94) segments clipped to [10,400], start time uniform integer in
    [0, 300-len], own window [t0,t1] drawn uniformly inside its extent, own d
    uniform in [0.5,10].  `box` is the edge of the start cube (1000)."""
    rng = np.random.default_rng(seed)
    counts = np.full(n_traj, n_points, np.int64)
    starts = rng.uniform(0.0, box, size=(n_traj, 3))
    pts = _walk_points(starts, counts, _exp_isotropic_steps(rng, int(counts.sum())))
    ent = polylines_to_segments(pts, _unit_times(np.zeros(n_traj), counts), counts, np.arange(n_traj))

    nseg = np.clip(np.round(rng.lognormal(np.log(63.2), 0.94, size=n_queries)), 10,
                   min(400, n_points - 1)).astype(np.int64)
    qstart = np.floor(rng.uniform(0.0, 1.0, size=n_queries) * (n_points - 1 - nseg + 1)).astype(np.int64)
    qcounts = nseg + 1
    qpos = rng.uniform(0.0, box, size=(n_queries, 3))
    qpts = _walk_points(qpos, qcounts, _exp_isotropic_steps(rng, int(qcounts.sum())))
    qry = polylines_to_segments(qpts, _unit_times(qstart.astype(np.float64), qcounts), qcounts,
                                np.arange(n_queries) + 10_000_000, first_seg_id=1 << 40)
    lo = qstart.astype(np.float64)
    hi = (qstart + nseg).astype(np.float64)
    u = np.sort(rng.uniform(0.0, 1.0, size=(n_queries, 2)), axis=1)
    w0 = lo + u[:, 0] * (hi - lo)
    w1 = lo + u[:, 1] * (hi - lo)
    dq = rng.uniform(0.5, 10.0, size=n_queries)
    rep = nseg
    return Workload("batching_walks", ent, qry, (), (float(ent.ts.min()), float(ent.te.max())),
                    q_d=np.repeat(dq, rep), q_t0=np.repeat(w0, rep), q_t1=np.repeat(w1, rep),
                    n_query_traj=n_queries, meta={"query_traj_segments": nseg})


def serving_database(seed=DEFAULT_SEED, n_traj=40_000, n_points=500) -> Segments:
    """Resident database: 40,000 walks x 500 points starting at t=0, steps
    Normal(0,1) per axis, start uniform in [0,1000]^3 (19.96 M segments)."""
    rng = np.random.default_rng(seed)
    counts = np.full(n_traj, n_points, np.int64)
    starts = rng.uniform(0.0, 1000.0, size=(n_traj, 3))
    pts = _walk_points(starts, counts, rng.standard_normal(size=(int(counts.sum()), 3)))
    return polylines_to_segments(pts, _unit_times(np.zeros(n_traj), counts), counts, np.arange(n_traj))


@dataclass
class Request:
    arrival_s: float
    query: Segments
    d: float
    t0: float
    t1: float


def serving_requests(seed=DEFAULT_SEED, n_requests=20_000, rate_per_s=2_000.0, n_points=500,
                     min_seg=5, max_seg=500):
    """Poisson arrivals at rate_per_s; each request is a fresh walk of
    min_seg..max_seg segments at a random integer start time inside the
    database extent [0, n_points-1], its own d uniform in [1,20] and its own
    window drawn inside its extent."""
    rng = np.random.default_rng(seed + 1)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    arrivals = np.cumsum(gaps)
    out = []
    base = 1 << 41
    for k in range(n_requests):
        ns = int(rng.integers(min_seg, min(max_seg, n_points - 1) + 1))
        t0 = float(rng.integers(0, n_points - 1 - ns + 1))
        pts = _walk_points(rng.uniform(0.0, 1000.0, size=(1, 3)), [ns + 1],
                           rng.standard_normal(size=(ns + 1, 3)))
        q = polylines_to_segments(pts, t0 + np.arange(ns + 1, dtype=np.float64), [ns + 1], [k],
                                  first_seg_id=base + k * 1024)
        u = np.sort(rng.uniform(0.0, 1.0, size=2))
        w0 = t0 + u[0] * ns
        w1 = t0 + u[1] * ns
        out.append(Request(float(arrivals[k]), q, float(rng.uniform(1.0, 20.0)), w0, w1))
    return out


def random_segments(rng, n, box=10.0, t_span=10.0, max_dur=2.0, max_speed=1.0) -> Segments:
    """Unstructured random segments (for small edge-case tests): start in
    [0,box]^3, start time in [0,t_span], duration in (0,max_dur], velocity
    components uniform in [-max_speed, max_speed]."""
    ts = rng.uniform(0.0, t_span, size=n)
    dur = rng.uniform(0.05, 1.0, size=n) * max_dur
    te = ts + dur
    p0 = rng.uniform(0.0, box, size=(n, 3))
    v = rng.uniform(-max_speed, max_speed, size=(n, 3))
    p1 = p0 + v * dur[:, None]
    return Segments(p0[:, 0].copy(), p0[:, 1].copy(), p0[:, 2].copy(), ts, p1[:, 0].copy(), p1[:, 1].copy(),
                    p1[:, 2].copy(), te, np.arange(n, dtype=np.int64), np.arange(n, dtype=np.int64))
