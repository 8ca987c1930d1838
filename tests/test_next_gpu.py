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


def _both_active(oracle_mod, mk, seed):
    """An equilibrated model (quench, then Langevin MD) with sigma and epsilon
    both inside their bands (the eigenvalue bias of Eq. 13 and Eq. 15)."""
    from paper_0909_5215_gb300 import model as M
    base = mk()
    o = oracle_mod.OracleReplica(base, M.Params())
    xq, _, _ = o.quench(method=1, ftol=1e-8, max_iter=20000)
    r = base.copy()
    r.pos, r.pos_ref, r.rep_id = xq.copy(), xq.copy(), seed
    o = oracle_mod.OracleReplica(r, M.Params())
    o.run(1000)
    r.pos, r.vel = o.x.copy(), o.v.copy()
    o = oracle_mod.OracleReplica(r, M.Params(bias_on=1))
    s0 = o.s.sigma
    e0, _ = o.lowest_eig()
    r.dvmax, r.m_exp, r.eig_on = 0.3, 2, 1
    r.sig_lo, r.sig_hi = s0 - 0.5 * abs(s0) - 0.1, s0 + 0.5 * abs(s0) + 0.1
    r.eig_lo, r.eig_hi = e0 - 0.5 * abs(e0) - 0.05, e0 + 0.5 * abs(e0) + 0.05
    return r


@pytest.mark.parametrize("prec", [0, 1])
def test_eigenvalue_bias_matches_oracle(hd, oracle_mod, prec):
    """Eq. 13 with DeltaV_2(epsilon) of Eq. 15: epsilon from Lanczos on the
    constrained Hessian, its gradient from phi''', in a batch with a plain
    slope-bias replica.  Both sides stop Lanczos at a Ritz residual of
    1e-10 |epsilon| (the GPU reorthogonalises by two passes of classical
    Gram-Schmidt where the oracle uses modified Gram-Schmidt), so epsilon
    agrees to ~1e-10 and the eigenvector, which enters the force through
    grad epsilon, to ~1e-10 over the spectral gap.  Tolerances: epsilon and
    DeltaV relative 1e-9 (FP64 form) / 1e-6 (split form) at the start and after
    30 steps; positions 1e-8 / 1e-4."""
    from paper_0909_5215_gb300 import model as M
    reps = [_both_active(oracle_mod, small2d, seed=11), _both_active(oracle_mod, small3d, seed=12)]
    plain = reps[0].copy()
    plain.eig_on, plain.rep_id = 0, 13
    reps.append(plain)
    p = M.Params(prec=prec, bias_on=1)
    b = hd.Batch(reps, p)
    ors = [oracle_mod.OracleReplica(r, p) for r in reps]
    rel = 1e-9 if prec == 0 else 1e-6
    for k, o in enumerate(ors):
        ob = b.obs(k)
        if reps[k].eig_on:
            assert 0.0 < o.s.dV2 < 0.3 and o.s.dVe != 0.0
            assert ob["eig"] == pytest.approx(o.s.eig, rel=1e-9)
            assert ob["eig_iters"] > 10
        assert ob["dV"] == pytest.approx(o.s.dV, rel=rel)
    th0 = [o.s.t_h for o in ors]
    b.step(30)
    oracle_mod.run_batch(ors, 30)
    for k, o in enumerate(ors):
        ob = b.obs(k)
        if reps[k].eig_on:
            assert ob["eig"] == pytest.approx(o.s.eig, rel=rel)
        assert ob["dV"] == pytest.approx(o.s.dV, rel=rel, abs=1e-12)
        assert ob["t_h"] - th0[k] == pytest.approx(o.s.t_h - th0[k], rel=rel)
        assert np.abs(b.positions(k) - o.x).max() < (1e-8 if prec == 0 else 1e-4)
    b.close()


def test_eigenvalue_bias_keeps_the_per_phase_driver(hd, oracle_mod):
    """A batch with the eigenvalue bias asks for the persistent driver and
    gets the per-phase kernels (the Lanczos runs one CTA per replica)."""
    from paper_0909_5215_gb300 import model as M
    r = thermalise(small2d(), amp=0.03, seed=61)
    r.eig_on, r.eig_lo, r.eig_hi, r.dvmax = 1, -1.0, 1.0, 0.2
    b = hd.Batch([r], M.Params(prec=1, bias_on=1), driver=hd.HD_DRIVER_PERSISTENT)
    assert b.info()["driver"] == hd.HD_DRIVER_KERNELS
    b.step(5)
    b.sync()
    b.close()
