"""Pins of the restart-schedule checks (oracle/schedule.py) used by the GPU
parity tests: they must accept the rule's own schedule and reject a
schedule that breaks Algorithm alg-apg-re's spacing or takes a decision the
other way where d_t is not a rounding-level tie."""
import numpy as np
import pytest

import oracle
from oracle import schedule as S
import synth


def _poisson(N):
    Q, b, _ = synth.workload("poisson2d_%d" % N)
    return Q, b, oracle.j_absrowsum(Q)


def test_spacing_rule():
    S.check_spacing([], 2)
    S.check_spacing([3, 8, 17], 2)          # 3 > 0 + 2, 8 > 3 + 4, 17 > 8 + 8
    for bad in ([2], [3, 7], [3, 8, 16], [5, 4]):
        with pytest.raises(S.ScheduleError):
            S.check_spacing(bad, 2)
    S.check_spacing([11], 10)
    with pytest.raises(S.ScheduleError):
        S.check_spacing([10], 10)
    with pytest.raises(S.ScheduleError):
        S.check_spacing([40], 2, restart=False)


def test_natural_schedule_replays_without_flips():
    Q, b, J = _poisson(32)
    T = 400
    nat, ref = S.natural(Q, b, T, J=J)
    assert len(nat) >= 3
    S.check_spacing(nat, 2)
    rep = S.replay(Q, b, nat, T, J=J)
    assert rep["flips"] == []
    np.testing.assert_array_equal(rep["x"], ref["x"])


def test_natural_schedule_of_the_64x64_solve_has_no_near_tie():
    # the case the GPU must reproduce exactly: 2-D Poisson 64 x 64 to 1e-12
    Q, b, J = _poisson(64)
    ref = oracle.solve(Q, b, J, tol=1e-12, maxit=20000, trace=True)
    tr = ref["trace"]
    sched = [int(t) for t in np.nonzero(tr["restart"])[0]]
    assert len(sched) >= 3
    ratio = np.abs(tr["d"][1:]) / (tr["gnorm"][1:] * tr["dxnorm"][1:])
    assert ratio.min() > 1e-6  # every decision is 6 orders above the guard


@pytest.mark.parametrize("mutate", ["late", "early", "extra", "dropped", "off_by_one_rule"])
def test_planted_schedule_mistakes_are_rejected(mutate):
    Q, b, J = _poisson(32)
    T = 400
    nat, _ = S.natural(Q, b, T, J=J)
    t1 = nat[0]
    if mutate == "late":         # the first restart one iteration late
        bad = [t1 + 1] + nat[1:]
    elif mutate == "early":      # one iteration early (d < 0 there, or the spacing breaks)
        bad = [t1 - 1] + nat[1:]
    elif mutate == "extra":      # a restart where the rule continues
        bad = nat[:1] + [nat[1] - 5] + nat[1:]
    elif mutate == "dropped":    # a restart left out
        bad = nat[1:]
    else:
        # t >= K_re + K instead of t > K_re + K: with K_0 = 64 the oracle's d is
        # already >= 0 at t = 64 (clearly, not a tie), so that rule restarts at
        # 64 where alg-apg-re waits until 65
        nat64, _ = S.natural(Q, b, 200, J=J, K0=64)
        assert nat64 == [65, 200]
        with pytest.raises(S.ScheduleError):
            S.replay(Q, b, [64], 200, J=J, K0=64)
        return
    with pytest.raises(S.ScheduleError):
        S.replay(Q, b, sorted(bad), T, J=J)


def test_tie_within_the_guard_is_accepted():
    # a zero right-hand side from x^0 = 0: x stays 0, d = 0 = ||g|| ||dx||, and a
    # restart there is a tie in either direction
    Q, b, J = _poisson(8)
    z = np.zeros_like(b)
    nat, _ = S.natural(Q, z, 40, J=J)
    assert nat == [3, 8, 17, 34]  # d = 0 >= 0: a tie restarts as soon as the spacing allows
    for sched in ([3], [], [3, 8, 17, 34]):
        rep = S.replay(Q, z, sched, 40, J=J)
        assert np.all(rep["x"] == 0.0)
