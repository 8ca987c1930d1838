"""Parallel stepped sliding (Sec. 2.3, Fig. 2): host logic on the CPU.

A scripted batch (clock rates, transition times and F_R per slider position)
pins the bookkeeping: the smallest position with a transition wins, later
positions are discarded, the next interval restarts from the transition
state with the rest of that period, transitions after a period's end do not
count, time adds up, and F_R is averaged over boosted time.  A batch backed
by the oracle then drives a small 2-D model through a real slip.
"""
import numpy as np
import pytest

from conftest import small2d
from oracle_batch import OracleBatch

DT = 0.005
OBS_LEN = 24


class ScriptedBatch:
    """Replica at slider index j: t_h grows by alpha[j] dt per MD step, a
    transition is flagged once t_h >= T[j], F_R reads fr[j], the slope sigma
    reads 10 j + (MD steps so far) / 1000; set_bias calls are recorded."""

    def __init__(self, reps, params, x0, dx, alpha, T, fr):
        self.idx = [int(round((r.slider[0] - x0) / dx)) for r in reps]
        self.n = [r.n for r in reps]
        self.th = np.zeros(len(reps))
        self.steps = 0
        self.alpha, self.T, self.fr = alpha, T, fr
        self.bias = []
        self.closed = False

    def step(self, n):
        self.th += n * DT * np.array([self.alpha.get(j, 1.0) for j in self.idx])
        self.steps += n

    def obs(self):
        ob = np.zeros((len(self.idx), OBS_LEN))
        ob[:, 2] = self.th
        ob[:, 6] = [10.0 * j + self.steps / 1000.0 for j in self.idx]
        ob[:, 8] = [self.fr.get(j, 0.0) for j in self.idx]
        return ob

    def set_bias(self, bias):
        self.bias.append(np.asarray(bias, dtype=np.float64).reshape(len(self.idx), 4).copy())

    def quench(self, theta=0.5, adopt=0, **kw):
        return np.array([int(self.th[k] >= self.T.get(j, np.inf)) for k, j in enumerate(self.idx)], dtype=np.int32)

    def _tag(self, k, what):
        return np.full((self.n[k], 3), 1000.0 * what + self.idx[k])

    def positions(self, k):
        return self._tag(k, 1)

    def velocities(self, k):
        return self._tag(k, 2)

    def qpos(self, k):
        return self._tag(k, 3)

    def ref(self, k):
        return self._tag(k, 4)

    def close(self):
        self.closed = True


def _driver(alpha=None, T=None, fr=None, n_par=4, dtau=1.0, check_every=50, **kw):
    from paper_0909_5215_gb300 import model as M
    from paper_0909_5215_gb300.sliding import SteppedSliding
    st = small2d()
    st.pos_ref = st.pos.copy()
    dx = 0.1
    x0 = float(st.slider[0])
    made = []

    def mk(reps, params):
        b = ScriptedBatch(reps, params, x0, dx, alpha or {}, T or {}, fr or {})
        made.append(b)
        return b

    d = SteppedSliding(st, M.Params(prec=1), dx=dx, v_s=dx / dtau, n_par=n_par, check_every=check_every,
                       make_batch=mk, **kw)
    return d, made


def test_no_transition_accepts_every_position():
    d, made = _driver()
    assert d.interval() is None
    assert d.m == 4 and d.t_in == 0.0 and d.time == pytest.approx(4.0)
    assert [p.index for p in d.log.periods] == [0, 1, 2, 3]
    assert all(p.time == pytest.approx(1.0) and not p.transition for p in d.log.periods)
    assert np.all(d.state.pos == 1003.0) and np.all(d.state.pos_ref == 4003.0)   # last replica's state
    assert d.state.slider[0] == pytest.approx(d.x0[0] + 0.4)
    assert made[0].closed


def test_smallest_transition_wins_and_restarts_there():
    # checks every 0.25 of boosted time; index 3 slips first, index 2 later
    d, _ = _driver(T={2: 0.6, 3: 0.3})
    assert d.interval() == 2
    assert [p.index for p in d.log.periods] == [0, 1, 2]
    assert d.log.periods[2].transition and d.log.periods[2].time == pytest.approx(0.75)
    assert d.time == pytest.approx(2.75) and d.t_in == pytest.approx(0.75)
    assert d.log.transitions == [(2, pytest.approx(d.x0[0] + 0.2), pytest.approx(2.75))]
    # the new state is replica 2's state when flagged, r_O its quenched minimum
    assert np.all(d.state.pos == 1002.0) and np.all(d.state.vel == 2002.0) and np.all(d.state.pos_ref == 3002.0)
    # the next interval starts at index 2 with the rest of that period
    d.interval()
    assert d.log.periods[3].index == 2 and d.log.periods[3].time == pytest.approx(0.25)
    assert d.time == pytest.approx(sum(p.time for p in d.log.periods))


def test_later_transition_at_a_lower_position_takes_over():
    d, _ = _driver(T={1: 0.9, 3: 0.2})
    assert d.interval() == 1
    assert [p.index for p in d.log.periods] == [0, 1]
    assert d.time == pytest.approx(1.0 + 1.0)    # flagged at the check at t_h = 1.0


def test_transition_after_the_period_ended_does_not_count():
    # index 0 would slip at 1.1, after its period (1.0); index 1 runs at half
    # speed, so the interval goes on past that time
    d, _ = _driver(alpha={1: 0.5}, T={0: 1.1}, n_par=2)
    assert d.interval() is None
    assert d.m == 2 and d.time == pytest.approx(2.0)


def test_boosted_clock_and_f_r_average():
    d, _ = _driver(alpha={0: 4.0, 1: 1.0}, fr={0: 0.3, 1: 0.5}, n_par=2)
    d.interval()
    assert [p.fr_mean for p in d.log.periods] == [pytest.approx(0.3), pytest.approx(0.5)]
    assert d.time == pytest.approx(2.0)
    with pytest.raises(ValueError):
        _driver(n_par=0)


def test_basin_lost_at_a_position_is_a_transition_at_its_start():
    # the quench that sets r_O at each position already leaves the basin at
    # index 2: a transition at time 0 of that period
    d, _ = _driver(T={2: 0.0, 3: 0.0})
    assert d.interval() == 2
    assert [p.index for p in d.log.periods] == [0, 1, 2]
    assert d.log.periods[2].transition and d.log.periods[2].time == 0.0
    assert d.time == pytest.approx(2.0) and d.t_in == 0.0
    # without the requench the first check finds it, a check interval later
    d, _ = _driver(T={2: 0.0, 3: 0.0}, requench=False)
    assert d.interval() == 2
    assert d.log.periods[2].time == pytest.approx(0.25)


def test_transition_that_closes_a_period_moves_to_the_next_position():
    # flagged at the check where index 0's period ends (t_h = 1.0)
    d, _ = _driver(T={0: 1.0}, n_par=2)
    assert d.interval() == 0
    assert d.t_in == pytest.approx(1.0)
    d.interval()
    # no empty period at index 0: the next interval starts at index 1
    assert [p.index for p in d.log.periods] == [0, 1, 2]
    assert all(p.time > 0 for p in d.log.periods)


def test_band_prerun_sets_each_replica_band_from_its_own_slopes():
    band = dict(prerun=200, sample_every=50, q_lo=0.25, q_hi=0.75, dvmax=0.3, m=3)
    d, made = _driver(n_par=3, band=band)
    d.interval()
    b = made[0]
    assert len(b.bias) == 2
    assert np.all(b.bias[0][:, 0] == 0.0)                 # the pre-run is unbiased
    # slopes sampled after 50, 100, 150, 200 steps: 10 j + {0.05 .. 0.2}
    samples = np.array([0.05, 0.1, 0.15, 0.2])
    for j in range(3):
        dvmax, lo, hi, m = b.bias[1][j]
        assert (dvmax, m) == (0.3, 3.0)
        assert lo == pytest.approx(10 * j + np.quantile(samples, 0.25))
        assert hi == pytest.approx(10 * j + np.quantile(samples, 0.75))
    # the pre-run is MD at the position and counts toward the period: it
    # fills the 200-step periods, and one check follows it
    assert d.log.md_steps == 200 + 50
    assert d.time == pytest.approx(3.0)
    with pytest.raises(ValueError):
        _driver(band=dict(q_lo=0.6, q_hi=0.5))


def test_f_r_is_sampled_between_checks():
    # F_R changes only through which replica is read; sampling every 10 steps
    # gives the same boosted average as sampling at the checks
    d, _ = _driver(alpha={0: 4.0, 1: 1.0}, fr={0: 0.3, 1: 0.5}, n_par=2, sample_every=10)
    d.interval()
    assert [p.fr_mean for p in d.log.periods] == [pytest.approx(0.3), pytest.approx(0.5)]
    with pytest.raises(ValueError):
        _driver(sample_every=30)


def _log(rows):
    from paper_0909_5215_gb300.sliding import Period, SlidingLog
    lg = SlidingLog()
    for i, f, t in rows:
        lg.periods.append(Period(index=i, slider_x=0.1 * i, time=1.0, fr_mean=f, transition=t))
    return lg


def test_slip_forces_stick_phases_windows_and_hops():
    from paper_0909_5215_gb300.sliding import slip_forces
    rows = [(0, 1.0, False), (1, 3.0, False), (2, 2.0, False), (3, 2.5, True),    # slip at 3, peak 3.0
            (3, 9.0, False), (4, 1.0, False), (5, 1.5, False), (6, 2.0, True),    # peak 9.0 right after the slip
            (7, 0.5, True),                                                      # second hop of the same slip
            (8, 1.0, False), (9, float("nan"), True)]                            # nan periods are skipped
    lg = _log(rows)
    assert slip_forces(lg) == [(3, 3.0), (6, 9.0), (7, 0.5), (9, 1.0)]
    assert slip_forces(lg, min_gap=2) == [(3, 3.0), (6, 9.0), (9, 1.0)]
    # the last 3 periods only: the relaxation after the previous slip drops out
    assert slip_forces(lg, min_gap=2, window=3) == [(3, 3.0), (6, 2.0), (9, 1.0)]


class ScriptedSlider:
    """Moving-slider batch: F_R = 2 x travel; a replica flags a transition
    at the first check after its slider has travelled past each of `slips`."""

    def __init__(self, reps, params, slips):
        self.v = [r.v_slide for r in reps]
        self.dt = params.dt
        self.steps = 0
        self.slips = slips
        self.done = [set() for _ in reps]
        self.adopts = []

    def step(self, n):
        self.steps += n

    def obs(self):
        ob = np.zeros((len(self.v), OBS_LEN))
        ob[:, 0] = self.steps
        ob[:, 1] = self.steps * self.dt
        ob[:, 8] = [2.0 * v * self.dt * self.steps for v in self.v]
        return ob

    def quench(self, theta=0.5, adopt=0, **kw):
        self.adopts.append(adopt)
        out = []
        for k, v in enumerate(self.v):
            hit = [x for x in self.slips if v * self.dt * self.steps >= x and x not in self.done[k]]
            self.done[k].update(hit)
            out.append(int(bool(hit)))
        return np.array(out, dtype=np.int32)

    def close(self):
        pass


def test_continuous_sliding_bins_and_dates_transitions():
    from paper_0909_5215_gb300 import model as M
    from paper_0909_5215_gb300.sliding import ContinuousSliding, slip_forces
    st = small2d()
    p = M.Params(prec=1, dt=0.005)
    made = []

    def mk(reps, params):
        b = ScriptedSlider(reps, params, slips=[0.53, 1.01])
        made.append(b)
        return b

    # bins of 0.1003 sigma: no sample falls on a bin edge
    cs = ContinuousSliding(st, p, v_s=0.01, n_samples=2, dx=0.1003, sample_every=100, check_every=400,
                           make_batch=mk)
    logs = cs.run(1.2)
    b = made[0]
    assert all(v == 0.01 for v in b.v) and set(b.adopts) == {1}
    for lg in logs:
        assert lg.md_steps == 24000
        # a sample every 0.005 sigma of travel; bin i holds travel in [0.1003 i, 0.1003 (i + 1))
        assert [q.index for q in lg.periods] == list(range(12))
        assert lg.periods[0].fr_mean == pytest.approx(2.0 * np.mean(np.arange(1, 21) * 0.005))
        assert all(q.time == pytest.approx(10.03) for q in lg.periods)
        # checks every 0.02 of travel: the slips are dated at 0.54 and 1.02
        assert [t[0] for t in lg.transitions] == [5, 10]
        assert [t[1] - st.slider[0] for t in lg.transitions] == [pytest.approx(0.54), pytest.approx(1.02)]
        assert [i for i, _ in slip_forces(lg)] == [5, 10]
    with pytest.raises(ValueError):
        ContinuousSliding(st, M.Params(prec=1, bias_on=1), v_s=0.01, n_samples=1, dx=0.1, make_batch=mk)


def test_oracle_backed_sliding_through_a_slip(oracle_mod):
    """A small 2-D tip dragged 0.15 sigma per period with four positions in
    flight: the spring loads until the tip slips by a lattice spacing, the
    slip is flagged, and the run restarts from the slipped state."""
    from paper_0909_5215_gb300 import model as M
    from paper_0909_5215_gb300.sliding import SteppedSliding
    base = small2d(kT=0.02)
    p = M.Params(prec=0, bias_on=0)
    o = oracle_mod.OracleReplica(base, p)
    xq, _, _ = o.quench(method=1, ftol=1e-6, max_iter=20000)
    st = base.copy()
    st.pos, st.pos_ref = xq.copy(), xq.copy()
    d = SteppedSliding(st, p, dx=0.15, v_s=0.15 / 0.5, n_par=4, check_every=50, theta=0.5,
                       quench=dict(method=1, ftol=1e-4, max_iter=3000),
                       make_batch=lambda reps, params: OracleBatch(reps, params, oracle_mod))
    rig = st.role == 2
    x_tip0 = float(st.pos[rig, 0].mean())
    for _ in range(12):
        d.interval()
        if d.log.transitions:
            break
    assert d.log.transitions, "no slip within 12 intervals"
    assert d.time == pytest.approx(sum(p.time for p in d.log.periods))
    # the adopted basin is the quenched state after the slip: its rigid layer
    # moved forward by more than theta from where it started
    assert float(d.state.pos_ref[rig, 0].mean()) - x_tip0 > 0.5
    # loading before the slip: F_R grows with the slider position
    frs = [p.fr_mean for p in d.log.periods if not p.transition]
    assert len(frs) >= 2 and frs[-1] > frs[0]


def test_ensemble_in_one_batch_equals_separate_runs(oracle_mod):
    """Three samples (own states and replica ids, one seed) run together in
    one oracle-backed batch per interval give exactly the logs and states of
    three separate runs: a sample whose interval ends early (a slip) stops
    counting and carries on from its state at that moment."""
    from paper_0909_5215_gb300 import model as M
    from paper_0909_5215_gb300.sliding import SteppedSliding, run_ensemble, run_intervals
    base = small2d(kT=0.02)
    p = M.Params(prec=0, bias_on=0, seed=5)
    xq, _, _ = oracle_mod.OracleReplica(base, p).quench(method=1, ftol=1e-6, max_iter=20000)
    mk = lambda reps, params: OracleBatch(reps, params, oracle_mod)

    def drivers():
        out = []
        for s in range(3):
            st = base.copy()
            st.pos, st.pos_ref, st.rep_id = xq.copy(), xq.copy(), 50 + s
            o = oracle_mod.OracleReplica(st, p)
            o.run(200 + 100 * s)
            st.pos, st.vel = o.x.copy(), o.v.copy()
            out.append(SteppedSliding(st, p, dx=0.2, v_s=0.4, n_par=4, check_every=100, sample_every=20,
                                      quench=dict(method=1, ftol=1e-4, max_iter=3000), make_batch=mk,
                                      rep_id0=1000 * (s + 1)))
        return out

    together, apart = drivers(), drivers()
    run_ensemble(together, 16)
    for d in apart:
        while d.m < 16:
            d.interval()
    assert sum(len(d.log.transitions) for d in apart) >= 1
    for a, t in zip(apart, together):
        assert t.m == a.m and t.time == a.time and t.t_in == a.t_in
        assert t.log.md_steps == a.log.md_steps and t.log.intervals == a.log.intervals
        assert t.log.transitions == a.log.transitions
        assert [(q.index, q.time, q.transition) for q in t.log.periods] == \
               [(q.index, q.time, q.transition) for q in a.log.periods]
        assert np.array_equal([q.fr_mean for q in t.log.periods], [q.fr_mean for q in a.log.periods], equal_nan=True)
        assert np.array_equal(t.state.pos, a.state.pos) and np.array_equal(t.state.pos_ref, a.state.pos_ref)
    # drivers with different settings cannot share a batch
    d1, d2 = drivers()[:2]
    d2.check_every = 200
    with pytest.raises(ValueError):
        run_intervals([d1, d2])
