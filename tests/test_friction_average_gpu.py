"""Time-averaged lateral force F_R = k (x_S - x_T) (Eq. 10) over a long run.

Two 421-atom 2-D replicas (48x8 substrate, 37-atom tip, T = 0.05) held at
slider offsets of 0.2 and 0.5 sigma, bias on (DeltaV_max = 4 kT, band from
the 5% and 50% quantiles of sigma in an oracle pre-run).  From one state the
split-form GPU batch and the FP64 oracle each run 20,000 steps (100 tau) and
sample F_R and DeltaV every 100 steps.  Both the plain time average of F_R
and the boost-weighted one (weights exp(beta DeltaV), the hyperdynamics
estimate of the unbiased time average) must agree within 2%.  Both sides
draw the same Philox noise, so the trajectories stay together and the
agreement is far inside the bound; the bound itself allows for trajectories
that separate, as chaotic ones do over longer runs.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

STEPS, EVERY = 20000, 100


@pytest.fixture(scope="module")
def hd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_5215_gb300 import _build, hd as H
    _build.build()
    return H


def _states(oracle_mod):
    from paper_0909_5215_gb300 import model as M
    base = M.afm2d(kT=0.05, eps=M.PAPER_EPS_2D)
    p = M.Params(prec=1, bias_on=1)
    o = oracle_mod.OracleReplica(base, p)
    xq, _, _ = o.quench(method=1, ftol=1e-6, max_iter=20000)
    out = []
    for k, off in enumerate((0.2, 0.5)):
        r = base.copy()
        r.pos, r.pos_ref = xq.copy(), xq.copy()
        r.rep_id = 40 + k
        r.slider = r.slider + np.array([off, 0.0])
        o = oracle_mod.OracleReplica(r, p)
        sig = []
        for _ in range(20):
            o.run(100)
            sig.append(o.s.sigma)
        st = r.copy()
        st.pos, st.vel = o.x.copy(), o.v.copy()
        st.t_h0, st.t_md0, st.step0 = o.s.t_h, o.s.t_md, int(o.s.step)
        st.dvmax, st.m_exp = 4.0 * st.kT, 2
        st.sig_lo, st.sig_hi = float(np.quantile(sig, 0.05)), float(np.quantile(sig, 0.5))
        out.append(st)
    return out, p


def _averages(fr, dv, kT):
    fr, w = np.asarray(fr), np.exp(np.asarray(dv) / kT)
    return fr.mean(), (fr * w).sum() / w.sum()


def test_time_averaged_friction_force_within_2_percent(hd, oracle_mod):
    reps, p = _states(oracle_mod)
    b = hd.Batch(reps, p)
    iF, iV = hd.OBS_FIELDS.index("F_R"), hd.OBS_FIELDS.index("dV")
    g_fr, g_dv = [], []
    for _ in range(STEPS // EVERY):
        b.step(EVERY)
        ob = b.obs()
        g_fr.append(ob[:, iF].copy())
        g_dv.append(ob[:, iV].copy())
    b.close()
    g_fr, g_dv = np.array(g_fr), np.array(g_dv)
    for k, r in enumerate(reps):
        o = oracle_mod.OracleReplica(r, p)
        o_fr, o_dv = [], []
        for _ in range(STEPS // EVERY):
            o.run(EVERY)
            o_fr.append(o.s.FR)
            o_dv.append(o.s.dV)
        assert max(o_dv) > 0.0                               # the bias was active
        g_plain, g_boost = _averages(g_fr[:, k], g_dv[:, k], r.kT)
        o_plain, o_boost = _averages(o_fr, o_dv, r.kT)
        assert abs(g_plain - o_plain) <= 0.02 * abs(o_plain)
        assert abs(g_boost - o_boost) <= 0.02 * abs(o_boost)
