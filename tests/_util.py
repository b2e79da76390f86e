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


def compare_results(gpu, ora, entries, queries, d, t0=-np.inf, t1=np.inf, dmin_fn=None,
                    d_per_query=None, win_per_query=None):
    """Compare two result sets keyed by (query index, entry index).

    gpu / ora: dicts with arrays 'qi', 'ei', 't_enter', 't_exit'.
    Pairs present on one side only must be ties (|dmin - d| <= TIE_REL * d),
    checked with dmin_fn(ei, qi) supplied by the caller (the oracle).  Matched
    pairs must agree on both endpoints within ENDPOINT_REL * max(1, |t|),
    unless the endpoint is ill-conditioned, in which case the reported time
    must still put the pair at distance d within the same relative band.
    Returns a dict of counts."""
    def key(r):
        return r["qi"].astype(np.int64) * (1 << 32) + r["ei"].astype(np.int64)

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
        dd = d if d_per_query is None else float(d_per_query[qi])
        dm = dmin_fn(ei, qi)
        assert np.isfinite(dm) and abs(dm - dd) <= TIE_REL * dd, (
            f"pair (q={qi}, e={ei}) reported by one side only; dmin={dm!r}, d={dd!r}")
        ties += 1
    bad = 0
    max_rel = 0.0
    for name in ("t_enter", "t_exit"):
        a = gpu[name][og][ig]
        b = ora[name][oo][io]
        tol = ENDPOINT_REL * np.maximum(1.0, np.abs(b))
        if len(a):
            max_rel = max(max_rel, float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))))
        off = np.nonzero(np.abs(a - b) > tol)[0]
        for j in off:
            k = int(common[j])
            qi, ei = k >> 32, k & 0xFFFFFFFF
            dd = d if d_per_query is None else float(d_per_query[qi])
            e8 = entries.row(ei)
            q8 = queries.row(qi)
            dist = float(dist_at(e8, q8, a[j])[0])
            assert abs(dist - dd) <= TIE_REL * dd + 1e-12, (
                f"{name} mismatch for pair (q={qi}, e={ei}): {a[j]!r} vs {b[j]!r}, dist at ours {dist!r}")
            bad += 1
    return {"matched": len(common), "ties": ties, "ill_conditioned_endpoints": bad, "max_endpoint_rel": max_rel,
            "gpu_only": len(only_g), "oracle_only": len(only_o)}
