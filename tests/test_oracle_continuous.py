"""Oracle pins for continuous sliding (Sec. 3.1.1, method 1: the slider moves
every step at v_S instead of being stepped).

The slider's x after k steps is x_S0 + k (v_S dt), written out exactly; with
v_S = 0 the run is the stepped-sliding one bit for bit; and in NVE the work
theorem holds: the potential depends on time only through x_S, so
d(K + V)/dt = (dV/dx_S) v_S = F_R v_S (Eq. 10), and K + V - int F_R v_S dt is
conserved up to an integration error ~ dt^2.
"""
import numpy as np
import pytest

from conftest import small2d


def _params(**kw):
    from paper_0909_5215_gb300 import model as M
    return M.Params(**kw)


@pytest.fixture(scope="module")
def state(oracle_mod):
    base = small2d()
    o = oracle_mod.OracleReplica(base, _params())
    xq, _, _ = o.quench(method=1, ftol=1e-8, max_iter=20000)
    r = base.copy()
    r.pos, r.pos_ref = xq.copy(), xq.copy()
    o = oracle_mod.OracleReplica(r, _params())
    o.run(1000)
    st = r.copy()
    st.pos, st.vel = o.x.copy(), o.v.copy()
    return st


def test_slider_position_is_exact(oracle_mod, state):
    s = state.copy()
    s.v_slide = 0.01
    o = oracle_mod.OracleReplica(s, _params())
    x0 = float(s.slider[0])
    o.run(250)
    assert o.s.slider[0] == x0 + 250.0 * (0.01 * 0.005)
    assert o.s.slider[1] == s.slider[1]


def test_zero_velocity_is_stepped_sliding(oracle_mod, state):
    a = oracle_mod.OracleReplica(state.copy(), _params())
    s = state.copy()
    s.v_slide = 0.0
    b = oracle_mod.OracleReplica(s, _params())
    a.run(200)
    b.run(200)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) and a.s.FR == b.s.FR


def test_work_theorem_second_order(oracle_mod, state):
    v = 0.5
    devs = []
    for dt in (0.004, 0.002):
        s = state.copy()
        s.gamma, s.v_slide = 0.0, v
        o = oracle_mod.OracleReplica(s, _params(dt=dt))
        e0, w, fr, dev = o.s.K + o.s.V, 0.0, o.s.FR, 0.0
        for _ in range(int(round(1.0 / dt))):
            o.run(1)
            w += 0.5 * (fr + o.s.FR) * v * dt           # trapezoid of F_R v_S dt
            fr = o.s.FR
            dev = max(dev, abs(o.s.K + o.s.V - e0 - w))
        devs.append(dev)
        assert abs(w) > 10 * dev                          # the work is resolved
    assert devs[0] < 5e-3
    assert 3.0 < devs[0] / devs[1] < 5.0
