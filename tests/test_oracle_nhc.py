"""Oracle pins for the Nose-Hoover chain thermostat (Sec. 3.1.1).

The chain (Martyna-Tuckerman-Tobias-Klein reversible splitting) must conserve
the extended energy K + V (+ DeltaV) + sum Q v^2/2 + N_f kT xi_1 + kT sum xi_j
with an error ~ dt^2, hold the mobile atoms at the set temperature
(<m v^2> = kT per degree of freedom), and reduce to plain NVE dynamics when
its masses are very large.
"""
import numpy as np
import pytest

from conftest import small2d


def _params(**kw):
    from paper_0909_5215_gb300 import model as M
    return M.Params(**kw)


@pytest.fixture(scope="module")
def state(oracle_mod):
    base = small2d(kT=0.1)
    o = oracle_mod.OracleReplica(base, _params())
    xq, _, _ = o.quench(method=1, ftol=1e-8, max_iter=20000)
    r = base.copy()
    r.pos, r.pos_ref = xq.copy(), xq.copy()
    o = oracle_mod.OracleReplica(r, _params())
    o.run(1000)
    st = r.copy()
    st.pos, st.vel = o.x.copy(), o.v.copy()
    st.nhc_len, st.nhc_tau = 3, 0.5
    return st


@pytest.mark.parametrize("bias", [0, 1])
def test_extended_energy_second_order(oracle_mod, state, bias):
    s0 = state.copy()
    if bias:
        o = oracle_mod.OracleReplica(s0, _params(bias_on=1))
        sg = o.s.sigma
        s0.dvmax, s0.sig_lo, s0.sig_hi = 0.3, 0.5 * sg, 1.5 * sg
    devs = []
    for dt in (0.004, 0.002):
        o = oracle_mod.OracleReplica(s0.copy(), _params(dt=dt, bias_on=bias))
        e0, dev = o.s.K + o.s.V + o.s.dV + o.nhc_energy(), 0.0
        for _ in range(5):
            o.run(int(round(0.2 / dt)))
            dev = max(dev, abs(o.s.K + o.s.V + o.s.dV + o.nhc_energy() - e0))
        assert o.nhc_energy() != 0.0                      # the chain took part
        devs.append(dev)
    assert devs[0] < 5e-3
    assert 3.0 < devs[0] / devs[1] < 5.0


def test_holds_the_temperature(oracle_mod, state):
    o = oracle_mod.OracleReplica(state.copy(), _params())
    mob = state.role == 1
    nf = 2 * int(mob.sum())
    t = []
    for _ in range(800):
        o.run(50)
        t.append(float((o.v[mob, :2] ** 2).sum()) / nf)
    assert np.mean(t) == pytest.approx(state.kT, rel=0.05)


def test_heavy_chain_is_plain_nve(oracle_mod, state):
    s = state.copy()
    s.nhc_tau = 1e6                                       # masses ~ 1e12: the chain barely moves
    a = oracle_mod.OracleReplica(s, _params())
    n = state.copy()
    n.nhc_len, n.gamma = 0, 0.0
    b = oracle_mod.OracleReplica(n, _params())
    a.run(200)
    b.run(200)
    assert np.abs(a.v - b.v).max() < 1e-8 and np.abs(a.x - b.x).max() < 1e-9
