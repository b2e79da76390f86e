"""Shared helpers for the tests: golden-file parsing, independent position
evaluation, and comparison of two result sets under the tie rule."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# A pair whose true distance of closest approach lies within this relative
# band of d is a tie: the two sides may decide it differently.
TIE_REL = 1e-9
# Matched interval endpoints agree to this relative tolerance.
ENDPOINT_REL = 1e-9


def read_golden(name):
    """Parse a golden text file into {section: [[floats...], ...]}."""
    sections, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = line[1:-1]
                sections[cur] = []
                continue
            sections[cur].append([float(x) for x in line.split()])
    return sections


def pos_at(seg8, t):
    """Position of a segment's moving point at time(s) t, by interpolating its
    endpoints with numpy (independent of the oracle's C code)."""
    seg8 = np.asarray(seg8, np.float64)
    t = np.asarray(t, np.float64)
    p0 = seg8[[0, 1, 2]]
    p1 = seg8[[4, 5, 6]]
    f = (t - seg8[3]) / (seg8[7] - seg8[3])
    return p0[None, :] + (p1 - p0)[None, :] * np.atleast_1d(f)[:, None]


def dist_at(e8, q8, t):
    return np.linalg.norm(pos_at(q8, t) - pos_at(e8, t), axis=1)


# Ill-conditioned endpoints allowed on the galaxy workload.  A root moves by
# about (rounding of the squared distance) / (slope there), and the slope at a
# root is 2 |dv| sqrt(d^2 - dmin^2): only pairs whose closest approach lies
# within ~1e-18 relative of d, i.e. ties in all but name, can move a root by
# more than 1e-9 relative.  Co-orbiting stars come close to that; random
# walks never do, so there the allowance is zero.
GALAXY_ILL_CONDITIONED_MAX = 4


def common_span(entries, queries, qi, ei, t0=-np.inf, t1=np.inf):
    """[a, b]: the common time span of each (query qi, entry ei) pair inside
    the window, from the segments' end times (Sec. 3; numpy, independent of
    both sides).  t0 / t1 are scalars or per-pair arrays."""
    a = np.maximum(np.maximum(np.asarray(entries["ts"])[ei], np.asarray(queries["ts"])[qi]), t0)
    b = np.minimum(np.minimum(np.asarray(entries["te"])[ei], np.asarray(queries["te"])[qi]), t1)
    return a, b


def _min_dist_between(e8, q8, ta, tb):
    """Smallest distance of the pair over the time interval between ta and tb
    (the relative position is linear in t, so the closest point of that chord
    to the origin)."""
    pa = pos_at(q8, ta)[0] - pos_at(e8, ta)[0]
    pb = pos_at(q8, tb)[0] - pos_at(e8, tb)[0]
    w = pb - pa
    ww = float(w @ w)
    s = 0.0 if ww == 0.0 else min(1.0, max(0.0, -float(pa @ w) / ww))
    return float(np.linalg.norm(pa + s * w))


def compare_results(gpu, ora, entries, queries, d, t0=-np.inf, t1=np.inf, dmin_fn=None,
                    d_per_query=None, win_per_query=None, max_ill_conditioned=0):
    """Compare two result sets keyed by (query index, entry index).

    gpu / ora: dicts with arrays 'qi', 'ei', 't_enter', 't_exit'.

    - Every GPU interval lies inside the pair's common span clipped to the
      window, in order: a <= t_enter <= t_exit <= b (Sec. 3: the result is a
      sub-interval of the time both segments are defined and the window
      allows).  The span is recomputed here from the inputs.
    - Pairs present on one side only must be ties (|dmin - d| <= TIE_REL * d),
      checked with dmin_fn(ei, qi) supplied by the caller (the oracle).
    - Matched pairs agree on both endpoints within ENDPOINT_REL * max(1, |t|).
      An endpoint outside that band is accepted only as an ill-conditioned
      root: the pair is at distance d within TIE_REL * d at the GPU's time, the
      GPU's time lies on the oracle's side of the interval (t_enter not past
      the oracle's t_exit, t_exit not before its t_enter), and between the two
      times the distance never drops below d (1 - TIE_REL), so both name the
      same root of the quadratic (calcTimeInterval, Sec. 5) and not the other
      one.  At most max_ill_conditioned endpoints may take this branch.

    win_per_query: optional (t0 array, t1 array) indexed by query, overriding
    t0 / t1.  Returns a dict of counts."""
    def key(r):
        return r["qi"].astype(np.int64) * (1 << 32) + r["ei"].astype(np.int64)

    def window_of(qi):
        if win_per_query is None:
            return t0, t1
        return np.asarray(win_per_query[0])[qi], np.asarray(win_per_query[1])[qi]

    def d_of(qi):
        return d if d_per_query is None else float(d_per_query[qi])

    gq = np.asarray(gpu["qi"], np.int64)
    ge = np.asarray(gpu["ei"], np.int64)
    gin = np.asarray(gpu["t_enter"], np.float64)
    gout = np.asarray(gpu["t_exit"], np.float64)
    if len(gq):
        w0, w1 = window_of(gq)
        a, b = common_span(entries, queries, gq, ge, w0, w1)
        # a + tau rounds to at most half an ulp of (b - a) past b
        slack = 4 * np.finfo(np.float64).eps * np.maximum(np.abs(a), np.abs(b))
        bad = ~((a < b) & np.isfinite(gin) & np.isfinite(gout) & (a <= gin) & (gin <= gout + slack)
                & (gout <= b + slack))
        if np.any(bad):
            j = int(np.nonzero(bad)[0][0])
            raise AssertionError(
                f"GPU interval of pair (q={gq[j]}, e={ge[j]}) is not inside its common span: "
                f"[{gin[j]!r}, {gout[j]!r}] vs span [{a[j]!r}, {b[j]!r}] ({int(bad.sum())} such rows)")

    kg, ko = key(gpu), key(ora)
    assert len(np.unique(kg)) == len(kg), "duplicate pair in the GPU result"
    assert len(np.unique(ko)) == len(ko), "duplicate pair in the oracle result"
    og, oo = np.argsort(kg), np.argsort(ko)
    kg, ko = kg[og], ko[oo]
    common, ig, io = np.intersect1d(kg, ko, assume_unique=True, return_indices=True)
    only_g = np.setdiff1d(kg, ko, assume_unique=True)
    only_o = np.setdiff1d(ko, kg, assume_unique=True)
    ties = 0
    for k in np.concatenate([only_g, only_o]):
        qi, ei = int(k >> 32), int(k & 0xFFFFFFFF)
        dd = d_of(qi)
        dm = dmin_fn(ei, qi)
        assert np.isfinite(dm) and abs(dm - dd) <= TIE_REL * dd, (
            f"pair (q={qi}, e={ei}) reported by one side only; dmin={dm!r}, d={dd!r}")
        ties += 1
    ga = {n: np.asarray(gpu[n], np.float64)[og][ig] for n in ("t_enter", "t_exit")}
    oa = {n: np.asarray(ora[n], np.float64)[oo][io] for n in ("t_enter", "t_exit")}
    ill = 0
    max_rel = 0.0
    for name, other in (("t_enter", "t_exit"), ("t_exit", "t_enter")):
        g, o = ga[name], oa[name]
        tol = ENDPOINT_REL * np.maximum(1.0, np.abs(o))
        if len(g):
            max_rel = max(max_rel, float(np.max(np.abs(g - o) / np.maximum(1.0, np.abs(o)))))
        off = np.nonzero(np.abs(g - o) > tol)[0]
        for j in off:
            k = int(common[j])
            qi, ei = k >> 32, k & 0xFFFFFFFF
            dd = d_of(qi)
            e8 = entries.row(ei)
            q8 = queries.row(qi)
            dist = float(dist_at(e8, q8, g[j])[0])
            assert abs(dist - dd) <= TIE_REL * dd + 1e-12, (
                f"{name} mismatch for pair (q={qi}, e={ei}): {g[j]!r} vs {o[j]!r}, dist at ours {dist!r}")
            # the same root: on the oracle's side of the interval ...
            if name == "t_enter":
                assert g[j] <= oa[other][j] + tol[j], (
                    f"t_enter of pair (q={qi}, e={ei}) lies past the oracle's t_exit: {g[j]!r} > {oa[other][j]!r}")
            else:
                assert g[j] >= oa[other][j] - tol[j], (
                    f"t_exit of pair (q={qi}, e={ei}) lies before the oracle's t_enter: {g[j]!r} < {oa[other][j]!r}")
            # ... with no dip inside d between the two times
            dm = _min_dist_between(e8, q8, min(g[j], o[j]), max(g[j], o[j]))
            assert dm >= dd * (1 - TIE_REL) - 1e-12, (
                f"{name} of pair (q={qi}, e={ei}) is on the other root: {g[j]!r} vs {o[j]!r}, the distance "
                f"drops to {dm!r} < d={dd!r} between them")
            ill += 1
    assert ill <= max_ill_conditioned, (
        f"{ill} ill-conditioned endpoints, more than the {max_ill_conditioned} allowed for this workload")
    return {"matched": len(common), "ties": ties, "ill_conditioned_endpoints": ill, "max_endpoint_rel": max_rel,
            "gpu_only": len(only_g), "oracle_only": len(only_o)}
