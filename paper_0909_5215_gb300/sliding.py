"""Stepped sliding with the slider positions of one interval run in parallel.

Sec. 2.3 replaces continuous sliding by a slider that jumps by dx_S after
each period dtau = dx_S / v_S, frozen in between (Fig. 1).  With a bias of
boost alpha the transition probability of one period is reached after
dtau / alpha of simulated time (Eq. 8), so each period ends when the
replica's boosted clock t_h (Eq. 3) reaches dtau.  When the slider moves
slowly enough for the system to equilibrate at every position, the periods
at successive positions are independent and can run at the same time
(Fig. 2): n_par replicas start from the current state at positions
x_m, ..., x_{m+n_par-1}.  If a transition occurs, the result of the smallest
position with a transition stands, every later position is discarded, and
the next interval starts from the state right after that transition.  (The
paper's "latest slider position that experienced a transition" is read as
the first one in slider order: only it is reached by the serial sequence of
periods.)  Without a transition all n_par periods are accepted and the next
interval starts at x_{m+n_par} from the state of the last replica.

The driver is host logic over a batch object with the calls of hd.Batch
(step, obs, quench, positions, velocities, qpos, ref, close); make_batch
builds one from replicas and parameters (hd.Batch by default).  Transitions
are checked every `check_every` MD steps by a quench (hd_quench, adopt = 0)
that flags a replica whose quenched minimum moved by more than theta from its
r_O.  A transition is dated at the boosted clock of the check that flags it
(resolution: one check interval) and counts when the replica's period was
still open at the previous check.  Periods that end inside a check interval
are cut at dtau for the time accounting and for the boost-weighted average
of F_R over the period, sampled at the checks (F_R times the t_h increment).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

OBS_T_H, OBS_DV, OBS_FR = 2, 5, 8       # columns of the OBS record


@dataclass
class Period:
    """One accepted period at one slider position."""
    index: int            # slider step count from the start
    slider_x: float
    time: float           # boosted time spent at this position in this period
    fr_mean: float        # F_R averaged over the period's boosted time
    transition: bool      # the period ended with a transition


@dataclass
class SlidingLog:
    periods: list = field(default_factory=list)
    transitions: list = field(default_factory=list)   # (index, slider_x, time of the transition)
    intervals: int = 0                                  # parallel intervals run
    md_steps: int = 0                                   # MD steps per replica, summed over intervals


class SteppedSliding:
    """Parallel stepped sliding (Fig. 2) over a batch of slider positions.

    state: a model.Replica at the current slider position with r_O
    (pos_ref) set to its current basin minimum and, for hyperdynamics, its
    bias band set.  dx: slider step dx_S; v_s: sliding velocity (dtau = dx /
    v_s); n_par: positions run at the same time.
    """

    def __init__(self, state, params, dx, v_s, n_par, check_every=500, theta=0.5,
                 quench=None, make_batch=None, max_checks=100000, rep_id0=1000):
        if dx <= 0 or v_s <= 0 or n_par < 1 or check_every < 1:
            raise ValueError("dx, v_s, n_par and check_every must be positive")
        self.state = state.copy()
        self.params = params
        self.dx = float(dx)
        self.dtau = float(dx) / float(v_s)
        self.n_par = int(n_par)
        self.check_every = int(check_every)
        self.theta = float(theta)
        self.quench = dict(method=1, ftol=1e-4, max_iter=2000) if quench is None else dict(quench)
        if make_batch is None:
            from . import hd
            make_batch = hd.Batch
        self.make_batch = make_batch
        self.max_checks = int(max_checks)
        self.x0 = np.array(state.slider, dtype=np.float64).copy()
        self.m = 0            # slider steps taken
        self.t_in = 0.0       # boosted time already spent at the current position
        self.time = 0.0       # boosted time since the start
        self.next_id = int(rep_id0)
        self.log = SlidingLog()

    def slider_at(self, index):
        return self.x0 + np.array([index * self.dx, 0.0])

    def _replicas(self):
        reps = []
        for k in range(self.n_par):
            r = self.state.copy()
            r.slider = self.slider_at(self.m + k)
            r.rep_id = self.next_id
            self.next_id += 1
            r.t_h0, r.t_md0, r.step0 = 0.0, 0.0, 0
            reps.append(r)
        return reps

    def interval(self):
        """Run one parallel interval; returns the first slider index with a
        transition in it, or None."""
        R = self.n_par
        budget = np.full(R, self.dtau)
        budget[0] = max(self.dtau - self.t_in, 0.0)
        reps = self._replicas()
        b = self.make_batch(reps, self.params)
        try:
            t_prev = np.zeros(R)
            t_tr = np.full(R, np.inf)          # boosted time of a counted transition
            fr_sum, t_sum = np.zeros(R), np.zeros(R)
            snap = {}
            kstar = None
            for _ in range(self.max_checks):
                b.step(self.check_every)
                self.log.md_steps += self.check_every
                ob = np.asarray(b.obs())
                th = ob[:, OBS_T_H]
                # boost-weighted F_R over each open period, cut at its end
                dt = np.clip(np.minimum(th, budget) - np.minimum(t_prev, budget), 0.0, None)
                dt[np.isfinite(t_tr)] = 0.0
                fr_sum += ob[:, OBS_FR] * dt
                t_sum += dt
                flags = np.asarray(b.quench(theta=self.theta, adopt=0, **self.quench))
                for k in range(R):
                    if flags[k] and not np.isfinite(t_tr[k]) and t_prev[k] < budget[k]:
                        t_tr[k] = min(th[k], budget[k])
                        snap[k] = (b.positions(k), b.velocities(k), b.qpos(k))
                t_prev = th.copy()
                hit = np.nonzero(np.isfinite(t_tr))[0]
                kstar = int(hit[0]) if hit.size else None
                upto = kstar if kstar is not None else R
                if all(th[k] >= budget[k] for k in range(upto)):
                    break
            else:
                raise RuntimeError("interval did not finish within max_checks quench checks")
            # accept periods [0, upto) in full and, with a transition, the
            # transition's period up to the transition
            for k in range(upto):
                self._period(k, budget[k], fr_sum[k], t_sum[k], False)
            if kstar is not None:
                self._period(kstar, t_tr[kstar], fr_sum[kstar], t_sum[kstar], True)
                x, v, xq = snap[kstar]
                self.time += budget[:kstar].sum() + t_tr[kstar]
                self.log.transitions.append((self.m + kstar, float(self.slider_at(self.m + kstar)[0]), self.time))
                self.t_in = (self.t_in if kstar == 0 else 0.0) + t_tr[kstar]
                self.m += kstar
                self.state.pos, self.state.vel, self.state.pos_ref = x, v, xq
            else:
                self.time += budget.sum()
                self.state.pos, self.state.vel = b.positions(R - 1), b.velocities(R - 1)
                self.state.pos_ref = b.ref(R - 1)
                self.m += R
                self.t_in = 0.0
            self.state.slider = self.slider_at(self.m)
            self.log.intervals += 1
            return None if kstar is None else self.m
        finally:
            b.close()

    def _period(self, k, t, fr_sum, t_sum, transition):
        self.log.periods.append(Period(index=self.m + k, slider_x=float(self.slider_at(self.m + k)[0]), time=float(t),
                                       fr_mean=float(fr_sum / t_sum) if t_sum > 0 else float("nan"),
                                       transition=transition))

    def run(self, n_positions):
        """Advance until the slider has taken n_positions steps."""
        target = self.m + int(n_positions)
        while self.m < target:
            self.interval()
        return self.log
