"""Checks of a restart schedule against the rule of Algorithm alg-apg-re
(Section 2.2), for the parity tests (TEST INFRASTRUCTURE ONLY).

The rule: iteration t restarts when IsRestart holds, t > K_re + K_ell and
d_t = <Q y^t - b, x^t - x^{t-1}> >= 0; a restart sets K_re = t and
K_{ell+1} = 2 K_ell, with K_0 given (K_re = 0 at the start).

The GPU and the oracle sum d_t in different orders, so when d_t sits at the
rounding level of its own scale ||Q y^t - b|| ||x^t - x^{t-1}|| (which bounds
|d_t| by Cauchy-Schwarz) the two may take opposite decisions.  Such a flip is
the only difference allowed:

* ``check_spacing`` asserts what the rule fixes whatever d is: restart
  iterations strictly increase and t_k > t_{k-1} + K_0 2^{k-1} (t_0 = 0), and
  there is none when IsRestart is off.
* ``replay`` runs the oracle with the given schedule forced and, at every
  iteration, evaluates the rule on the oracle's own d_t.  Wherever the rule
  decides otherwise than the schedule, |d_t| must be at most
  ``guard * ||Q y^t - b|| * ||x^t - x^{t-1}||`` (guard = 1e-12 by default);
  any other difference raises ``ScheduleError``.  Once the iteration has
  converged to the rounding level, Q y^t - b is itself rounding noise and
  so is the sign of d_t: the tie band then also admits
  |d_t| <= 64 (u + u_64) || |Q| |y^t| + |b| || ||x^t - x^{t-1}||, the
  rounding error a row sum of up to 64 terms can put into g in the GPU's
  unit roundoff u (2^-53 in FP64, 2^-48 in double-float) and the oracle's
  u_64 = 2^-53.  A schedule that passes is the rule's own up to
  rounding-level ties, and the returned oracle run is the trajectory the GPU
  must match.
* ``natural`` returns the oracle's own schedule, for tests that require the
  schedules to be equal outright.
"""
import numpy as np

from . import STOP_NONE, solve

GUARD = 1e-12
UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "df64": 2.0 ** -48}
FLOOR_TERMS = 64


class ScheduleError(AssertionError):
    pass


def check_spacing(sched, K0=2, restart=True):
    """The part of the restart rule that does not depend on d_t."""
    sched = [int(t) for t in sched]
    if not restart:
        if sched:
            raise ScheduleError("restarts %s with IsRestart off" % sched[:8])
        return
    prev, K = 0, int(K0)
    for k, t in enumerate(sched):
        if not t > prev + K:
            raise ScheduleError("restart %d at t = %d breaks t > K_re + K = %d + %d (schedule %s)"
                                % (k + 1, t, prev, K, sched[:12]))
        prev, K = t, 2 * K


def replay(Q, b, sched, T, *, J=None, Jblk=None, restart=True, momentum=True, K0=2, x0=None,
           guard=GUARD, precision="fp64"):
    """Oracle run of T iterations with the schedule forced, every decision of
    which is checked against the rule on the oracle's d_t (see the module
    docstring).  Returns the oracle's result dict plus ``flips``: the
    iterations where the schedule took the rounding-level tie the other way."""
    sched = sorted(int(t) for t in sched if 1 <= int(t) <= T)
    check_spacing(sched, K0, restart)
    ref = solve(Q, b, J, Jblk=Jblk, restart=restart, momentum=momentum, K0=K0, maxit=T,
                stop=STOP_NONE, x0=x0, forced=sched, trace=True)
    tr = ref["trace"]
    floor_unit = FLOOR_TERMS * (UNIT_ROUNDOFF[precision] + UNIT_ROUNDOFF["fp64"])
    S = set(sched)
    Kre, K = 0, int(K0)
    flips = []
    for t in range(1, ref["iters"] + 1):
        forced_t = t in S
        d = float(tr["d"][t])
        natural_t = bool(restart) and t > Kre + K and d >= 0.0
        if forced_t != natural_t:
            scale = float(tr["gnorm"][t]) * float(tr["dxnorm"][t])
            floor = floor_unit * float(tr["gfloor"][t]) * float(tr["dxnorm"][t])
            if not abs(d) <= guard * scale + floor:
                raise ScheduleError(
                    "iteration %d: schedule %s, rule on the oracle's d = %.3e says %s; "
                    "|d| / (||g|| ||dx||) = %.3e > %.0e, rounding floor %.3e" % (
                        t, "restarts" if forced_t else "continues", d,
                        "restart" if natural_t else "continue",
                        abs(d) / scale if scale > 0 else np.inf, guard, floor))
            flips.append(t)
        if forced_t:
            Kre, K = t, 2 * K
    ref["flips"] = flips
    return ref


def natural(Q, b, T, *, J=None, Jblk=None, restart=True, momentum=True, K0=2, x0=None):
    """The oracle's own restart iterations over T fixed iterations."""
    ref = solve(Q, b, J, Jblk=Jblk, restart=restart, momentum=momentum, K0=K0, maxit=T,
                stop=STOP_NONE, x0=x0, trace=True)
    return [int(t) for t in np.nonzero(ref["trace"]["restart"])[0]], ref
