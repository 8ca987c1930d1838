"""GPU parity of the rows after the hot path, through the C ABI, against the
CPU oracle.

Continuous sliding (Sec. 3.1.1, method 1): the slider moves along x at v_S
every step, x_S = x_S0 + k (v_S dt) for the configuration k steps after the
slider was set (closed form on both sides, so x_S is bit-identical).
Tolerances as for stepped sliding: positions 1e-9 (FP64 form) / 1e-4 (split
form) after 300 steps, F_R (Eq. 10) relative 1e-9 / 1e-5.
"""
import numpy as np
import pytest

from conftest import small2d, small3d, thermalise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_5215_gb300 import _build, hd as H
    _build.build()
    return H


@pytest.mark.parametrize("prec", [0, 1])
def test_continuous_sliding_matches_oracle(hd, oracle_mod, prec):
    from paper_0909_5215_gb300 import model as M
    reps = [thermalise(small2d(cols=16, rows=6, n_tip=13, kT=0.05), amp=0.03, seed=31),
            thermalise(small3d(nx=5, nz=3, radius=2.5, kT=0.08), amp=0.03, seed=32)]
    reps[0].v_slide, reps[1].v_slide = 0.05, -0.03
    reps[1].rep_id = 1
    p = M.Params(prec=prec, bias_on=0)
    b = hd.Batch(reps, p)
    ors = [oracle_mod.OracleReplica(r, p) for r in reps]
    b.step(100)
    b.step(50)
    oracle_mod.run_batch(ors, 150)
    xtol, ftol = (1e-9, 1e-9) if prec == 0 else (1e-4, 1e-5)
    for k, o in enumerate(ors):
        ob = b.obs(k)
        assert ob["x_S"] == o.s.slider[0]
        assert ob["x_S"] == reps[k].slider[0] + 150 * (reps[k].v_slide * p.dt)
        assert ob["F_R"] == pytest.approx(o.s.FR, rel=ftol, abs=1e-12)
        assert np.abs(b.positions(k) - o.x).max() < xtol
    # set the sliders again: the moving slider restarts from the new position
    new = np.array([[reps[0].slider[0] - 0.2, reps[0].slider[1]], [reps[1].slider[0] + 0.1, reps[1].slider[1]]])
    b.set_slider(new)
    for k, o in enumerate(ors):
        o.s.slider[0] = new[k, 0]
        o.s.slide_x0 = new[k, 0]
        o.s.slide_step0 = o.s.step
        o.refresh()
    b.step(150)
    oracle_mod.run_batch(ors, 150)
    for k, o in enumerate(ors):
        ob = b.obs(k)
        assert ob["x_S"] == o.s.slider[0]
        assert ob["F_R"] == pytest.approx(o.s.FR, rel=ftol, abs=1e-12)
        assert np.abs(b.positions(k) - o.x).max() < xtol
    b.close()


def test_continuous_sliding_persistent_driver(hd, oracle_mod):
    """The single-launch driver moves the slider the same way."""
    from paper_0909_5215_gb300 import model as M
    r = thermalise(small2d(cols=16, rows=6, n_tip=13, kT=0.05), amp=0.03, seed=33)
    r.v_slide = 0.04
    p = M.Params(prec=0, bias_on=0)
    b = hd.Batch([r], p, driver=hd.HD_DRIVER_PERSISTENT)
    o = oracle_mod.OracleReplica(r, p)
    b.step(120)
    o.run(120)
    ob = b.obs(0)
    assert ob["x_S"] == o.s.slider[0]
    assert np.abs(b.positions(0) - o.x).max() < 1e-9
    b.close()


def _bonded_models():
    from paper_0909_5215_gb300 import model as M
    r2 = M.paper2d(kT=0.02)
    r2.bonds = M.tip_bonds(r2)
    r3 = M.paper3d(kT=0.05)
    out = []
    for k, r in enumerate((r2, r3)):
        t = thermalise(r, amp=0.03, seed=40 + k)
        t.pos_ref = r.pos.copy()
        t.rep_id = k
        out.append(t)
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_tip_bonds_match_oracle(hd, oracle_mod, prec):
    """Harmonic tip bonds (Eq. 12, k = 57.2, r_b = 1.12) in place of tip-tip LJ:
    forces, H.(r - r_O) and energies, then 100 biased steps, against the oracle."""
    from paper_0909_5215_gb300 import model as M
    reps = _bonded_models()
    p = M.Params(prec=prec, bias_on=1)
    for r in reps:
        o = oracle_mod.OracleReplica(r, M.Params(prec=0, bias_on=0))
        s0 = o.s.sigma
        r.dvmax, r.sig_lo, r.sig_hi = 4.0 * r.kT, 0.7 * s0, 1.3 * s0
    b = hd.Batch(reps, p)
    ors = [oracle_mod.OracleReplica(r, p) for r in reps]
    tol = 1e-12 if prec == 0 else 1e-5

    def rms_rel(a, c):
        return float(np.sqrt(((a - c) ** 2).sum() / (c ** 2).sum()))

    for k, o in enumerate(ors):
        assert o.s.nbond > 0
        assert rms_rel(b.forces(k), o.f_lj) <= tol
        assert rms_rel(b.hdr(k), o.hdr) <= tol
        assert rms_rel(b.energies(k), o.e_atom) <= tol
        assert b.obs(k)["sigma"] == pytest.approx(o.s.sigma, rel=1e-12 if prec == 0 else 1e-6)
    b.step(100)
    oracle_mod.run_batch(ors, 100)
    for k, o in enumerate(ors):
        ob = b.obs(k)
        assert np.abs(b.positions(k) - o.x).max() < (1e-9 if prec == 0 else 1e-4)
        assert ob["t_h"] - reps[k].t_h0 == pytest.approx(o.s.t_h - reps[k].t_h0, rel=1e-9 if prec == 0 else 1e-6)
    b.close()


@pytest.mark.parametrize("prec,driver", [(0, 1), (1, 1), (0, 2)])
def test_nose_hoover_chain_matches_oracle(hd, oracle_mod, prec, driver):
    """Nose-Hoover chain (Sec. 3.1.1) in place of Langevin, mixed with a
    Langevin replica in one batch: positions, kinetic energy and the chain's
    energy after 200 steps against the oracle."""
    from paper_0909_5215_gb300 import model as M
    reps = [thermalise(small2d(cols=16, rows=6, n_tip=13, kT=0.05), amp=0.03, seed=51),
            thermalise(small3d(nx=5, nz=3, radius=2.5, kT=0.08), amp=0.03, seed=52),
            thermalise(small2d(cols=12, rows=6, n_tip=13, kT=0.05), amp=0.03, seed=53)]
    reps[0].nhc_len, reps[0].nhc_tau = 3, 0.5
    reps[1].nhc_len, reps[1].nhc_tau = 2, 0.8
    for k, r in enumerate(reps):
        r.rep_id = k
    p = M.Params(prec=prec, bias_on=0)
    b = hd.Batch(reps, p, driver=driver)
    ors = [oracle_mod.OracleReplica(r, p) for r in reps]
    b.step(120)
    b.step(80)
    oracle_mod.run_batch(ors, 200)
    xtol = 1e-9 if prec == 0 else 1e-4
    for k, o in enumerate(ors):
        ob = b.obs(k)
        assert np.abs(b.positions(k) - o.x).max() < xtol
        assert ob["K"] == pytest.approx(o.s.K, rel=1e-9 if prec == 0 else 1e-4)
        if reps[k].nhc_len:
            assert ob["nhc_energy"] == pytest.approx(o.nhc_energy(), rel=1e-9 if prec == 0 else 1e-4, abs=1e-12)
    b.close()
