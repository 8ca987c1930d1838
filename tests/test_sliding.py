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

DT = 0.005
OBS_LEN = 24


class ScriptedBatch:
    """Replica at slider index j: t_h grows by alpha[j] dt per MD step, a
    transition is flagged once t_h >= T[j], F_R reads fr[j]."""

    def __init__(self, reps, params, x0, dx, alpha, T, fr):
        self.idx = [int(round((r.slider[0] - x0) / dx)) for r in reps]
        self.n = [r.n for r in reps]
        self.th = np.zeros(len(reps))
        self.alpha, self.T, self.fr = alpha, T, fr
        self.closed = False

    def step(self, n):
        self.th += n * DT * np.array([self.alpha.get(j, 1.0) for j in self.idx])

    def obs(self):
        ob = np.zeros((len(self.idx), OBS_LEN))
        ob[:, 2] = self.th
        ob[:, 8] = [self.fr.get(j, 0.0) for j in self.idx]
        return ob

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


def _driver(alpha=None, T=None, fr=None, n_par=4, dtau=1.0, check_every=50):
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
                       make_batch=mk)
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


class OracleBatch:
    """The batch calls on the CPU oracle (test infrastructure only)."""

    def __init__(self, reps, params, oracle_mod):
        self.o = [oracle_mod.OracleReplica(r, params) for r in reps]
        self.xq = [o.x.copy() for o in self.o]

    def step(self, n):
        for o in self.o:
            o.run(n)

    def obs(self):
        ob = np.zeros((len(self.o), OBS_LEN))
        for k, o in enumerate(self.o):
            ob[k, 2], ob[k, 5], ob[k, 8] = o.s.t_h, o.s.dV, o.s.FR
        return ob

    def quench(self, method=1, ftol=1e-4, max_iter=2000, theta=0.5, adopt=0, step_size=None):
        flags = []
        for k, o in enumerate(self.o):
            xq, _, _ = o.quench(method=method, ftol=ftol, max_iter=max_iter)
            self.xq[k] = xq
            flags.append(int(o.transition(xq, theta)[0]))
        return np.array(flags, dtype=np.int32)

    def positions(self, k):
        return self.o[k].x.copy()

    def velocities(self, k):
        return self.o[k].v.copy()

    def qpos(self, k):
        return self.xq[k].copy()

    def ref(self, k):
        return self.o[k].xo.copy()

    def close(self):
        pass


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
