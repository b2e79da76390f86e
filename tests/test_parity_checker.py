"""The parity checker itself (tests/_util.compare_results), on the CPU.

Every GPU parity claim goes through compare_results, so it must reject the
mistakes a pair kernel could plausibly make while the distances at its
reported times still look right: an interval with its ends swapped, an
endpoint moved to the other root of the quadratic (both roots put the pair
at distance exactly d), and an interval that leaves the common span.  The
"GPU" results here are the oracle's own, altered by hand."""
import numpy as np
import pytest

from oracle import oracle
from paper_1405_7461_gb300 import workloads
from tests._util import compare_results


def _fly_by(beta, d=1.0):
    """One entry moving along x at unit speed through the origin at t = 10,
    one stationary query at distance beta from its path: in range for
    |t - 10| <= sqrt(d^2 - beta^2) (Sec. 3 with linear motion)."""
    ent = workloads.Segments.from_columns([np.array([v]) for v in (-10.0, 0.0, 0.0, 0.0, 10.0, 0.0, 0.0, 20.0)])
    qry = workloads.Segments.from_columns([np.array([v]) for v in (0.0, beta, 0.0, 0.0, 0.0, beta, 0.0, 20.0)])
    ref = oracle.search_bruteforce(ent, qry, d)
    assert len(ref.query_index) == 1
    ora = {"qi": ref.query_index, "ei": ref.entry_index, "t_enter": ref.t_enter, "t_exit": ref.t_exit}
    return ent, qry, ora


def _cmp(gpu, ora, ent, qry, d=1.0, **kw):
    return compare_results(gpu, ora, ent, qry, d,
                           dmin_fn=lambda ei, qi: oracle.pair_dmin(ent, ei, qry, qi), **kw)


def _with(ora, **times):
    g = {k: np.array(v, copy=True) for k, v in ora.items()}
    for k, v in times.items():
        g[k] = np.array([v], np.float64)
    return g


def test_fly_by_oracle_interval_is_the_closed_form():
    ent, qry, ora = _fly_by(0.5)
    h = np.sqrt(1.0 - 0.25)
    assert ora["t_enter"][0] == pytest.approx(10.0 - h, abs=1e-12)
    assert ora["t_exit"][0] == pytest.approx(10.0 + h, abs=1e-12)


def test_oracle_against_itself_passes():
    ent, qry, ora = _fly_by(0.5)
    c = _cmp(ora, ora, ent, qry)
    assert c["matched"] == 1 and c["ill_conditioned_endpoints"] == 0 and c["ties"] == 0


def test_swapped_endpoints_are_rejected():
    ent, qry, ora = _fly_by(0.5)
    g = _with(ora, t_enter=ora["t_exit"][0], t_exit=ora["t_enter"][0])
    with pytest.raises(AssertionError, match="not inside its common span"):
        _cmp(g, ora, ent, qry)


@pytest.mark.parametrize("moved", ["t_enter", "t_exit"])
def test_endpoint_on_the_other_root_is_rejected(moved):
    # the distance at the other root is d as well; only the dip between the
    # two roots tells them apart
    ent, qry, ora = _fly_by(0.5)
    other = "t_exit" if moved == "t_enter" else "t_enter"
    g = _with(ora, **{moved: ora[other][0]})
    with pytest.raises(AssertionError, match="other root"):
        _cmp(g, ora, ent, qry, max_ill_conditioned=10)


def test_endpoint_past_the_oracles_other_end_is_rejected():
    # t_enter reported beyond the oracle's t_exit, with t_exit moved along so
    # that the interval itself stays ordered
    ent, qry, ora = _fly_by(0.5)
    late = ora["t_exit"][0] + 0.25
    g = _with(ora, t_enter=late, t_exit=late + 0.1)
    with pytest.raises(AssertionError):
        _cmp(g, ora, ent, qry, max_ill_conditioned=10)


def test_interval_outside_the_common_span_is_rejected():
    ent, qry, ora = _fly_by(0.5)
    with pytest.raises(AssertionError, match="not inside its common span"):
        _cmp(_with(ora, t_exit=20.5), ora, ent, qry)
    with pytest.raises(AssertionError, match="not inside its common span"):
        _cmp(_with(ora, t_enter=-0.5), ora, ent, qry)
    # the window clips the span as well
    with pytest.raises(AssertionError, match="not inside its common span"):
        compare_results(ora, ora, ent, qry, 1.0, 0.0, 9.5, dmin_fn=lambda ei, qi: 0.0)


def test_per_query_window_clips_the_span():
    ent, qry, ora = _fly_by(0.5)
    with pytest.raises(AssertionError, match="not inside its common span"):
        _cmp(ora, ora, ent, qry, win_per_query=(np.array([0.0]), np.array([9.5])))
    c = _cmp(ora, ora, ent, qry, win_per_query=(np.array([0.0]), np.array([20.0])))
    assert c["matched"] == 1


def test_near_tangent_endpoint_on_the_same_root_is_accepted_and_counted():
    # impact parameter d (1 - 1e-12): the roots sit 1.4e-6 either side of the
    # closest point, the distance between them stays within 1e-9 d of d, so a
    # GPU endpoint moved halfway to the closest point is a valid root
    ent, qry, ora = _fly_by(1.0 - 1e-12)
    tin = ora["t_enter"][0]
    g = _with(ora, t_enter=tin + 0.5 * (10.0 - tin))
    c = _cmp(g, ora, ent, qry, max_ill_conditioned=1)
    assert c["ill_conditioned_endpoints"] == 1
    # ... and counted against the workload's allowance
    with pytest.raises(AssertionError, match="ill-conditioned"):
        _cmp(g, ora, ent, qry)


def test_one_sided_pair_must_be_a_tie():
    ent, qry, ora = _fly_by(0.5)
    empty = {k: v[:0] for k, v in ora.items()}
    with pytest.raises(AssertionError, match="one side only"):
        _cmp(empty, ora, ent, qry)
    # with the threshold at the closest distance, it is a tie
    ent, qry, ora = _fly_by(1.0 - 1e-13)
    c = _cmp(empty, ora, ent, qry)
    assert c["ties"] == 1
