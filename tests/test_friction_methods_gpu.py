"""Continuous, stepped and hyperdynamics stepped sliding on the GPU give the
same friction (Sec. 2.3, Sec. 3.1.2, Fig. 9): the acceptance of the parallel
stepped-sliding driver run through the library (hd.Batch, FP64 form, one
persistent launch per call).

The paper's 2-D model (Sec. 3.1.1: 80 substrate and 33 tip atoms, k = 5,
F_N = 5) at T = 0.01 is dragged at two fast sliding velocities, 1e-2 and
2e-3 sigma/tau, by three of the paper's four methods: continuous sliding,
parallel stepped sliding with the original potential, and with the slope
bias of Eq. 14 (dx_S = 0.05, 8 positions in flight, sigma_L and sigma_U from
a pre-run at each position).  At each velocity the lateral force at the
transitions (sliding.slip_forces) agrees between the methods within 5 % (at
1e-2) and 3 % (at 2e-3), and with the continuous-sliding force of the CPU
oracle's acceptance run of the same model within the same bounds (5.65 at
1e-2 and 5.31 at 2e-3, time averages over independent samples).  The force
falls as the velocity falls, and the bias spends fewer MD steps on the same
boosted time.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

T, DX, N_PAR = 0.01, 0.05, 8
A = 2.0 ** (1.0 / 6.0)
ORACLE_CONTINUOUS = {1e-2: 5.65, 2e-3: 5.31}     # the CPU acceptance run's means
BOUND = {1e-2: 0.05, 2e-3: 0.03}


@pytest.fixture(scope="module")
def hd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_5215_gb300 import _build, hd as H
    _build.build()
    return H


def _start(hd, base, xq, seed, steps=2000):
    """Equilibrate the quenched model for `steps` steps on the GPU."""
    from paper_0909_5215_gb300 import model as M
    r = base.copy()
    r.pos, r.pos_ref, r.rep_id = xq.copy(), xq.copy(), seed
    b = hd.Batch([r], M.Params(prec=0, bias_on=0, seed=seed), driver=hd.HD_DRIVER_PERSISTENT)
    b.step(steps)
    st = r.copy()
    st.pos, st.vel = b.positions(0), b.velocities(0)
    b.close()
    return st


def _methods(hd, v, distance, n_cont, n_step, check_every, prerun):
    from paper_0909_5215_gb300 import model as M
    from paper_0909_5215_gb300.sliding import ContinuousSliding, SteppedSliding, run_ensemble, slip_forces
    mk = lambda reps, params: hd.Batch(reps, params, driver=hd.HD_DRIVER_PERSISTENT)
    base = M.paper2d(kT=T)
    p0 = M.Params(prec=0, bias_on=0)
    b = hd.Batch([base], p0)
    b.quench(method=1, ftol=1e-8, max_iter=20000, step_size=0.01, theta=1e30, adopt=0)
    xq = b.qpos(0)
    b.close()
    gap = int(0.5 * A / DX)
    window = 5
    out = {}
    logs = ContinuousSliding(_start(hd, base, xq, 1), p0, v_s=v, n_samples=n_cont, dx=DX,
                             sample_every=50, check_every=check_every, make_batch=mk).run(distance)
    out["continuous"] = dict(logs=logs, forces=[slip_forces(lg, gap, window) for lg in logs])
    for name, bias in (("stepped", 0), ("hyper", 1)):
        p = M.Params(prec=0, bias_on=bias, seed=11)
        ds = [SteppedSliding(_start(hd, base, xq, s + 1), p, dx=DX, v_s=v, n_par=N_PAR,
                             check_every=check_every, sample_every=50,
                             quench=dict(method=1, ftol=1e-4, max_iter=3000), make_batch=mk,
                             rep_id0=(s + 1) * 100000,
                             band=dict(prerun=prerun, sample_every=10, dvmax=4 * T) if bias else None)
              for s in range(n_step)]
        n_pos = int(np.ceil(distance / DX))
        run_ensemble(ds, n_pos)
        out[name] = dict(logs=ds, forces=[slip_forces(d.log, gap, window) for d in ds])
    return out


def _mean(res):
    f = np.array([x for fs in res["forces"] for _, x in fs])
    return f.mean(), f.std() / np.sqrt(len(f)), len(f)


@pytest.fixture(scope="module")
def runs(hd):
    return {1e-2: _methods(hd, v=1e-2, distance=2.9, n_cont=8, n_step=4, check_every=500, prerun=400),
            2e-3: _methods(hd, v=2e-3, distance=3.9, n_cont=8, n_step=4, check_every=2000, prerun=2000)}


@pytest.mark.parametrize("v", [1e-2, 2e-3])
def test_methods_agree_on_the_force_at_transitions(runs, v):
    res = runs[v]
    fc, sc, nc = _mean(res["continuous"])
    report = ["v %.0e continuous %.3f +- %.3f (%d)" % (v, fc, sc, nc)]
    for name in ("stepped", "hyper"):
        f, s, n = _mean(res[name])
        report.append("%s %.3f +- %.3f (%d)" % (name, f, s, n))
    print("; ".join(report))
    assert nc >= 10, report
    assert abs(fc - ORACLE_CONTINUOUS[v]) <= BOUND[v] * ORACLE_CONTINUOUS[v], report
    for name in ("stepped", "hyper"):
        f, s, n = _mean(res[name])
        assert n >= 5, report
        assert abs(f - fc) <= BOUND[v] * fc, report


def test_friction_falls_with_velocity_and_bias_saves_steps(runs):
    assert _mean(runs[2e-3]["continuous"])[0] < _mean(runs[1e-2]["continuous"])[0] - 0.1
    for v in (1e-2, 2e-3):
        plain = sum(d.log.md_steps for d in runs[v]["stepped"]["logs"])
        hyper = sum(d.log.md_steps for d in runs[v]["hyper"]["logs"])
        assert hyper < plain, (v, hyper, plain)
