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

run_intervals and run_ensemble advance several independent runs (samples
with their own states and replica ids) together, one batch per interval
holding every sample's replicas; each sample's result is that of its own
run.

The driver is host logic over a batch object with the calls of hd.Batch
(step, obs, quench, positions, velocities, qpos, ref, close); make_batch
builds one from replicas and parameters (hd.Batch by default).  Transitions
are checked every `check_every` MD steps by a quench (hd_quench, adopt = 0)
that flags a replica whose quenched minimum moved by more than theta from its
r_O.  A transition is dated at the boosted clock of the check that flags it
(resolution: one check interval) and counts when the replica's period was
still open at the previous check.  Periods that end inside a check interval
are cut at dtau for the time accounting and for the boost-weighted average
of F_R over the period, sampled every `sample_every` steps (F_R times the
t_h increment).

The bias of Eq. 5 and Eq. 14 is measured from r_O, the minimum of the basin
the replica is in (after Eq. 7).  That minimum moves with the slider, so by
default every interval starts with a quench of each replica at its own slider
position that sets r_O (requench).  A replica whose quench already lands more
than theta from the carried r_O has lost its basin at that position: it makes
its transition at the start of its period.  With `band`, each replica also
runs an unbiased pre-run at its position and takes sigma_L and sigma_U as
quantiles of the slopes sampled there (the pre-simulation of Sec. 3.1.3); the
pre-run is ordinary MD and counts toward the period.

ContinuousSliding runs the reference method the stepped scheme replaces: the
slider moves at v_S every step (Sec. 3.1.1, method 1), F_R is averaged over
bins of slider travel dx, and the same quench test dates transitions.
slip_forces reads, from either log, the lateral force at each transition as
the largest period average of F_R at the end of the stick phase that ends
with it (the quantity the paper compares across methods, Sec. 3.1.2 and
Fig. 9).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

OBS_STEP, OBS_T_H, OBS_DV, OBS_SIGMA, OBS_FR = 0, 2, 5, 6, 8     # columns of the OBS record


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
    v_s); n_par: positions run at the same time.  requench: set r_O at each
    replica's own slider position when an interval starts.  band: None (keep
    the state's bias band) or a dict with prerun (MD steps), sample_every,
    q_lo, q_hi (quantiles of sigma for sigma_L, sigma_U), dvmax and m.
    sample_every: MD steps between F_R samples (a divisor of check_every).
    """

    def __init__(self, state, params, dx, v_s, n_par, check_every=500, theta=0.5,
                 quench=None, make_batch=None, max_checks=100000, rep_id0=1000,
                 requench=True, band=None, sample_every=None):
        sample_every = check_every if sample_every is None else sample_every
        if dx <= 0 or v_s <= 0 or n_par < 1 or check_every < 1 or sample_every < 1 or check_every % sample_every:
            raise ValueError("dx, v_s, n_par, check_every and sample_every must be positive, "
                             "check_every a multiple of sample_every")
        self.state = state.copy()
        self.params = params
        self.dx = float(dx)
        self.dtau = float(dx) / float(v_s)
        self.n_par = int(n_par)
        self.check_every = int(check_every)
        self.sample_every = int(sample_every)
        self.theta = float(theta)
        self.quench = dict(method=1, ftol=1e-4, max_iter=2000) if quench is None else dict(quench)
        if make_batch is None:
            from . import hd
            make_batch = hd.Batch
        self.make_batch = make_batch
        self.max_checks = int(max_checks)
        self.requench = bool(requench)
        self.band = None
        if band is not None:
            self.band = dict(prerun=2000, sample_every=20, q_lo=0.05, q_hi=0.5, dvmax=4.0 * state.kT, m=2)
            self.band.update(band)
            if not (0.0 <= self.band["q_lo"] < self.band["q_hi"] <= 1.0) or self.band["prerun"] < self.band["sample_every"]:
                raise ValueError("band: need 0 <= q_lo < q_hi <= 1 and prerun >= sample_every")
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
        return run_intervals([self])[0]

    def _settings(self):
        return (self.params, self.n_par, self.check_every, self.sample_every, self.theta, self.requench,
                tuple(sorted(self.quench.items())), None if self.band is None else tuple(sorted(self.band.items())),
                self.max_checks, self.make_batch)

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


class _Interval:
    """One driver's share of a batch during one interval: replicas
    [off, off + n_par) of the batch."""

    def __init__(self, d, off):
        R = d.n_par
        if d.t_in >= d.dtau:                # a transition closed the current position's period
            d.m += 1
            d.t_in = 0.0
            d.state.slider = d.slider_at(d.m)
        self.d, self.off, self.R = d, off, R
        self.budget = np.full(R, d.dtau)
        self.budget[0] = d.dtau - d.t_in
        self.reps = d._replicas()
        self.t_prev = np.zeros(R)           # boosted clocks at the last check
        self.t_acc = np.zeros(R)            # boosted clocks at the last F_R sample
        self.t_tr = np.full(R, np.inf)      # boosted time of a counted transition
        self.fr_sum, self.t_sum = np.zeros(R), np.zeros(R)
        self.snap = {}
        self.end = None                     # (x, v, r_O) of the last replica when done
        self.kstar, self.upto, self.done = None, R, False
        self.checks = 0

    def sl(self, a):
        return a[self.off:self.off + self.R]

    def flag(self, b, flags, th, at_start=False):
        for k in range(self.R):
            if flags[k] and not np.isfinite(self.t_tr[k]) and (at_start or self.t_prev[k] < self.budget[k]):
                self.t_tr[k] = 0.0 if at_start else min(th[k], self.budget[k])
                self.snap[k] = (b.positions(self.off + k), b.velocities(self.off + k), b.qpos(self.off + k))

    def accumulate(self, ob):
        # boost-weighted F_R over each open period, cut at its end
        th = ob[:, OBS_T_H]
        dt = np.clip(np.minimum(th, self.budget) - np.minimum(self.t_acc, self.budget), 0.0, None)
        dt[np.isfinite(self.t_tr)] = 0.0
        self.fr_sum += ob[:, OBS_FR] * dt
        self.t_sum += dt
        self.t_acc = th.copy()

    def settle(self, b, th):
        # the first position with a transition, the positions before it, and
        # whether all of those have used up their periods
        hit = np.nonzero(np.isfinite(self.t_tr))[0]
        self.kstar = int(hit[0]) if hit.size else None
        self.upto = self.kstar if self.kstar is not None else self.R
        self.done = all(th[k] >= self.budget[k] for k in range(self.upto))
        if self.done and self.kstar is None:
            last = self.off + self.R - 1
            self.end = (b.positions(last), b.velocities(last), b.ref(last))

    def finish(self):
        # accept periods [0, upto) in full and, with a transition, the
        # transition's period up to the transition
        d, kstar = self.d, self.kstar
        for k in range(self.upto):
            d._period(k, self.budget[k], self.fr_sum[k], self.t_sum[k], False)
        if kstar is not None:
            d._period(kstar, self.t_tr[kstar], self.fr_sum[kstar], self.t_sum[kstar], True)
            x, v, xq = self.snap[kstar]
            d.time += self.budget[:kstar].sum() + self.t_tr[kstar]
            d.log.transitions.append((d.m + kstar, float(d.slider_at(d.m + kstar)[0]), d.time))
            d.t_in = (d.t_in if kstar == 0 else 0.0) + self.t_tr[kstar]
            d.m += kstar
            d.state.pos, d.state.vel, d.state.pos_ref = x, v, xq
        else:
            d.time += self.budget.sum()
            d.state.pos, d.state.vel, d.state.pos_ref = self.end
            d.m += self.R
            d.t_in = 0.0
        d.state.slider = d.slider_at(d.m)
        d.log.intervals += 1
        return None if kstar is None else d.m


def run_intervals(drivers):
    """One interval of each SteppedSliding in `drivers`, all in one batch.

    The drivers are independent runs (samples, each its own state and
    replica ids) with the same settings.  Each keeps its own clocks, checks
    and result; a driver whose interval has finished stops counting while
    the others go on, and carries on from its state at that moment, so the
    result of each equals that of its own interval() whenever a replica's
    trajectory does not depend on the other replicas in the batch.  Returns
    each driver's interval() value."""
    if not drivers:
        return []
    d0 = drivers[0]
    if any(d._settings() != d0._settings() for d in drivers[1:]):
        raise ValueError("run_intervals: the drivers must share params, n_par, check/sample intervals, "
                         "theta, quench, requench, band, max_checks and make_batch")
    ivs, off = [], 0
    for d in drivers:
        ivs.append(_Interval(d, off))
        off += d.n_par
    b = d0.make_batch([r for iv in ivs for r in iv.reps], d0.params)
    try:
        zeros = np.zeros(off)
        if d0.requench:
            flags = np.asarray(b.quench(theta=d0.theta, adopt=2, **d0.quench))
            for iv in ivs:
                iv.flag(b, iv.sl(flags), None, at_start=True)
        for iv in ivs:
            iv.settle(b, iv.sl(zeros))
        if d0.band is not None and not all(iv.done for iv in ivs):
            _prerun(b, d0.band, [iv for iv in ivs if not iv.done], off)
        while not all(iv.done for iv in ivs):
            open_ = [iv for iv in ivs if not iv.done]
            for iv in open_:
                if iv.checks == d0.max_checks:
                    raise RuntimeError("interval did not finish within max_checks quench checks")
                iv.checks += 1
            for _ in range(d0.check_every // d0.sample_every):
                b.step(d0.sample_every)
                ob = np.asarray(b.obs())
                for iv in open_:
                    iv.d.log.md_steps += d0.sample_every
                    iv.accumulate(iv.sl(ob))
            th_all = ob[:, OBS_T_H]
            flags = np.asarray(b.quench(theta=d0.theta, adopt=0, **d0.quench))
            for iv in open_:
                th = iv.sl(th_all)
                iv.flag(b, iv.sl(flags), th)
                iv.t_prev = th.copy()
                iv.settle(b, th)
        return [iv.finish() for iv in ivs]
    finally:
        b.close()


def _prerun(b, band, open_, nrep):
    """Unbiased MD at every position, then sigma_L, sigma_U per replica
    from the slopes sampled during it (Eq. 14's band)."""
    m = float(band["m"])
    b.set_bias(np.tile([0.0, 0.0, 1.0, m], (nrep, 1)))
    n = int(band["prerun"]) // int(band["sample_every"])
    sig = np.empty((n, nrep))
    for i in range(n):
        b.step(int(band["sample_every"]))
        ob = np.asarray(b.obs())
        for iv in open_:
            iv.accumulate(iv.sl(ob))
        sig[i] = ob[:, OBS_SIGMA]
    for iv in open_:
        iv.d.log.md_steps += n * int(band["sample_every"])
    lo, hi = np.quantile(sig, band["q_lo"], axis=0), np.quantile(sig, band["q_hi"], axis=0)
    hi = np.maximum(hi, lo + 1e-12 * np.maximum(1.0, np.abs(lo)))
    b.set_bias(np.column_stack([np.full(nrep, float(band["dvmax"])), lo, hi, np.full(nrep, m)]))


def run_ensemble(drivers, n_positions):
    """Advance every driver until its slider has taken n_positions more
    steps, running the unfinished ones together interval by interval."""
    target = {id(d): d.m + int(n_positions) for d in drivers}
    while True:
        open_ = [d for d in drivers if d.m < target[id(d)]]
        if not open_:
            return [d.log for d in drivers]
        run_intervals(open_)


class ContinuousSliding:
    """Continuous sliding (Sec. 3.1.1, method 1) of n_samples independent
    replicas: the slider's x moves by v_s dt every MD step.

    state: a model.Replica with r_O (pos_ref) set to its basin minimum.
    Every `sample_every` steps F_R is read and added to the bin of slider
    travel dx it falls in; every `check_every` steps a quench (adopt = 1)
    flags the replicas that left their basin and moves their r_O to the new
    minimum.  The bias stays off: with the slider moving there is no frozen
    potential to boost.  The batch must support moving sliders (the replica
    field v_slide).
    """

    def __init__(self, state, params, v_s, n_samples, dx, sample_every=100, check_every=500, theta=0.5,
                 quench=None, make_batch=None, rep_id0=2000):
        if v_s <= 0 or n_samples < 1 or dx <= 0 or sample_every < 1 or check_every % sample_every:
            raise ValueError("v_s, n_samples, dx, sample_every must be positive; check_every a multiple of sample_every")
        if getattr(params, "bias_on", 0):
            raise ValueError("continuous sliding runs unbiased (bias_on = 0)")
        self.state = state.copy()
        self.params = params
        self.v_s, self.dx = float(v_s), float(dx)
        self.n_samples = int(n_samples)
        self.sample_every, self.check_every = int(sample_every), int(check_every)
        self.theta = float(theta)
        self.quench = dict(method=1, ftol=1e-4, max_iter=2000) if quench is None else dict(quench)
        if make_batch is None:
            from . import hd
            make_batch = hd.Batch
        self.make_batch = make_batch
        self.rep_id0 = int(rep_id0)
        self.x0 = float(state.slider[0])

    def run(self, distance):
        """Slide every sample by `distance`; returns one SlidingLog per sample
        with a Period per bin of slider travel dx."""
        dt = float(self.params.dt)
        nsteps = int(np.ceil(float(distance) / (self.v_s * dt) / self.sample_every)) * self.sample_every
        reps = []
        for k in range(self.n_samples):
            r = self.state.copy()
            r.rep_id = self.rep_id0 + k
            r.t_h0, r.t_md0, r.step0 = 0.0, 0.0, 0
            r.v_slide = self.v_s
            reps.append(r)
        nbin = int(np.ceil(float(distance) / self.dx)) + 1
        fr_sum = np.zeros((self.n_samples, nbin))
        cnt = np.zeros((self.n_samples, nbin))
        trans = [[] for _ in range(self.n_samples)]
        b = self.make_batch(reps, self.params)
        try:
            for done in range(self.sample_every, nsteps + 1, self.sample_every):
                b.step(self.sample_every)
                ob = np.asarray(b.obs())
                travel = self.v_s * dt * ob[:, OBS_STEP]
                j = np.minimum((travel / self.dx).astype(np.int64), nbin - 1)
                idx = np.arange(self.n_samples)
                fr_sum[idx, j] += ob[:, OBS_FR]
                cnt[idx, j] += 1
                if done % self.check_every == 0:
                    flags = np.asarray(b.quench(theta=self.theta, adopt=1, **self.quench))
                    for k in np.nonzero(flags)[0]:
                        trans[k].append((int(j[k]), self.x0 + float(travel[k]), float(ob[k, 1])))
        finally:
            b.close()
        logs = []
        tbin = self.dx / self.v_s
        for k in range(self.n_samples):
            lg = SlidingLog(md_steps=nsteps, intervals=1)
            hit = {t[0] for t in trans[k]}
            for i in range(nbin):
                if cnt[k, i] == 0:
                    continue
                lg.periods.append(Period(index=i, slider_x=self.x0 + i * self.dx, time=tbin,
                                         fr_mean=float(fr_sum[k, i] / cnt[k, i]), transition=i in hit))
            lg.transitions = trans[k]
            logs.append(lg)
        return logs


def slip_forces(log, min_gap=1, window=None):
    """The lateral force at each transition of a SlidingLog: the largest
    period average of F_R over the stick phase that the transition ends, or
    over its last `window` periods (the transition's own included), which
    keeps the relaxation right after the previous slip out.  Transitions
    fewer than min_gap slider positions after the previous one belong to
    the same slip (a slip in several hops) and end no new stick phase.
    Returns [(index of the transition, force)]."""
    out = []
    last = None
    cur = []
    for p in log.periods:
        cur.append(p.fr_mean)
        if not p.transition:
            continue
        if last is not None and p.index - last < min_gap:
            last = p.index
            cur = []
            continue
        vals = [v for v in (cur if window is None else cur[-int(window):]) if np.isfinite(v)]
        if vals:
            out.append((p.index, float(max(vals))))
        last = p.index
        cur = []
    return out
