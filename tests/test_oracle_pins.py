"""Pins of the CPU oracle against what the paper and the mathematics fix.

No GPU.  Each test checks the oracle against something other than itself:
published known-answer vectors, closed forms, brute force, finite
differences, conservation laws and special cases that reduce to plain MD.
"""
import os

import numpy as np
import pytest

from conftest import small2d, small3d, thermalise

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _params(**kw):
    from paper_0909_5215_gb300 import model as M
    return M.Params(**kw)


# ---------------------------------------------------------------- Philox
def test_philox_known_answers(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(t, 16) for t in row]
        assert oracle_mod.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_and_normals(oracle_mod):
    # the uniform lies strictly inside (0,1) at the extremes of the integer draw
    lib = oracle_mod.lib()
    assert lib.or_unif(0, 0) == 2.0 ** -53
    assert lib.or_unif(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert lib.or_unif(0x80000000, 0) == 0.5 + 2.0 ** -53
    # Box-Muller normals: mean 0, variance 1, independent pairs
    z = np.array([oracle_mod.normals(7, 3, s, a, 0) for s in range(200) for a in range(100)])
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.03
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.03


# ---------------------------------------------------------------- LJ, Eq. 9
def test_lj_closed_forms(oracle_mod):
    r0 = 2.0 ** (1.0 / 6.0)
    phi, dphi, d2phi = oracle_mod.lj(r0, rc=1e9)
    assert phi == pytest.approx(-1.0, abs=1e-14)          # minimum depth -eps
    assert abs(dphi) < 1e-13                               # zero force at 2^(1/6) sigma
    assert d2phi == pytest.approx(72.0 * 2.0 ** (-1.0 / 3.0), rel=1e-13)
    # paper: the harmonic tip bond of Eq. 12 (k = 57.2, r_O = 1.12) matches LJ at its minimum
    assert d2phi == pytest.approx(57.2, abs=0.06) and r0 == pytest.approx(1.12, abs=0.003)
    # shifted at rc = 2.5: phi(rc) = 0, minimum = -1 - phi_unshifted(2.5)
    assert oracle_mod.lj(2.5, rc=2.5)[0] == pytest.approx(0.0, abs=1e-16)
    p25 = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    assert p25 == pytest.approx(-0.0163169, abs=1e-7)
    assert oracle_mod.lj(r0, rc=2.5)[0] == pytest.approx(-1.0 - p25, abs=1e-14)
    # scaling: phi(r; eps, sig) = eps phi(r/sig; 1, 1)
    for eps, sig in ((0.5, 1.0), (0.2, 1.3)):
        a = oracle_mod.lj(1.4 * sig, eps, sig, 2.5 * sig)
        b = oracle_mod.lj(1.4, 1.0, 1.0, 2.5)
        assert a[0] == pytest.approx(eps * b[0], rel=1e-13)
        assert a[1] == pytest.approx(eps * b[1] / sig, rel=1e-13)
        assert a[2] == pytest.approx(eps * b[2] / sig ** 2, rel=1e-13)


def test_lj_derivatives_by_differences(oracle_mod):
    h = 1e-5
    for r in (0.95, 1.05, 1.3, 1.9, 2.4):
        p = oracle_mod.lj(r)
        pp, pm = oracle_mod.lj(r + h), oracle_mod.lj(r - h)
        assert (pp[0] - pm[0]) / (2 * h) == pytest.approx(p[1], rel=1e-8, abs=1e-9)
        assert (pp[1] - pm[1]) / (2 * h) == pytest.approx(p[2], rel=1e-7, abs=1e-8)


# ---------------------------------------------------------------- neighbour list
@pytest.mark.parametrize("mk", [small2d, small3d])
def test_nlist_cells_equals_brute(oracle_mod, mk):
    r = thermalise(mk(), amp=0.08)
    o = oracle_mod.OracleReplica(r, _params())
    o.nlist_brute()
    rb = o.rows()
    o.nlist_cells()
    rc = o.rows()
    assert all(np.array_equal(a, b) for a, b in zip(rb, rc))
    assert all(np.all(np.diff(a) > 0) for a in rb)          # strictly ascending j


def test_nlist_matches_independent_pair_search(oracle_mod):
    from scipy.spatial import cKDTree
    r = thermalise(small3d(), amp=0.08)
    o = oracle_mod.OracleReplica(r, _params())
    o.nlist_brute()
    rl = 2.8
    # periodic in x, y; the open axis is embedded in a box too large to wrap
    box = np.array([r.box[0], r.box[1], 1e6])
    pos = r.pos.copy()
    pos[:, 0] %= box[0]
    pos[:, 1] %= box[1]
    pos[:, 2] += 1e5
    pairs = cKDTree(pos, boxsize=box).query_pairs(rl, output_type="ndarray")
    got = {(i, j) for i in range(r.n) for j in o.rows()[i] if i < j}
    assert got == {(int(a), int(b)) for a, b in pairs}


def test_nlist_invariant_to_atom_order(oracle_mod):
    r = thermalise(small2d(), amp=0.08)
    o = oracle_mod.OracleReplica(r, _params())
    o.nlist_brute()
    ref = [set(x) for x in o.rows()]
    perm = np.random.default_rng(3).permutation(r.n)
    rp = r.copy()
    rp.pos, rp.role, rp.type = r.pos[perm], r.role[perm], r.type[perm]
    op = oracle_mod.OracleReplica(rp, _params())
    op.nlist_cells()
    rows = op.rows()
    for k in range(r.n):
        assert {int(perm[j]) for j in rows[k]} == ref[int(perm[k])]


# ---------------------------------------------------------------- forces, gradient, Hessian
@pytest.mark.parametrize("mk", [small2d, small3d])
def test_list_forces_equal_brute_force(oracle_mod, mk):
    r = thermalise(mk(), amp=0.06)
    o = oracle_mod.OracleReplica(r, _params())
    o.forces()
    fb, eb, vb = o.forces_brute()
    rms = np.sqrt(((o.f_lj - fb) ** 2).sum() / (fb ** 2).sum())
    assert rms < 1e-13
    assert o.s.V_lj == pytest.approx(vb, rel=1e-13)
    assert np.allclose(o.e_atom, eb, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("mk", [small2d, small3d])
def test_gradient_by_differences(oracle_mod, mk):
    r = thermalise(mk(), amp=0.06)
    o = oracle_mod.OracleReplica(r, _params())
    g = o.gradient()
    x = o.x.copy()
    h = 1e-5
    idx = list(range(0, r.n, max(1, r.n // 25))) + list(np.nonzero(r.role == 2)[0][:2])
    for i in idx:
        for a in range(r.dim):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = (o.potential(xp) - o.potential(xm)) / (2 * h)
            assert fd == pytest.approx(g[i, a], rel=1e-7, abs=1e-6)
    # the list-based LJ force is -grad of the LJ part
    o.forces()
    mob = r.role == 1
    assert np.allclose(-o.f_lj[mob], g[mob], rtol=1e-12, atol=1e-11)


@pytest.mark.parametrize("mk", [small2d, small3d])
def test_hessian_vector_by_differences(oracle_mod, mk):
    r = thermalise(mk(), amp=0.06)
    o = oracle_mod.OracleReplica(r, _params())
    rng = np.random.default_rng(0)
    u = rng.normal(size=(r.n, 3))
    w = rng.normal(size=(r.n, 3))
    for v in (u, w):
        v[r.role == 0] = 0.0
        if r.dim == 2:
            v[:, 2] = 0.0
    x = o.x.copy()
    h = 1e-5
    hu = o.hessvec(u)
    fd = (o.gradient(x + h * u) - o.gradient(x - h * u)) / (2 * h)
    assert np.abs(fd - hu).max() < 1e-6 * np.abs(hu).max()
    assert (u * o.hessvec(w)).sum() == pytest.approx((w * o.hessvec(u)).sum(), rel=1e-12)
    # the per-atom H.dr of the list-based sweep equals H applied to dr = x - x_O
    r2 = r.copy()
    r2.pos_ref = r.pos - 0.3 * u
    o2 = oracle_mod.OracleReplica(r2, _params())
    o2.forces()
    dr = o2.x - o2.xo
    assert np.allclose(o2.hdr, o2.hessvec(dr), rtol=1e-11, atol=1e-10)


# ---------------------------------------------------------------- bias, Eq. 14
def test_dv1_shape(oracle_mod):
    r = small2d()
    r.dvmax, r.sig_lo, r.sig_hi, r.m_exp = 0.4, 10.0, 20.0, 2
    o = oracle_mod.OracleReplica(r, _params(bias_on=1))
    assert tuple(o.dv1(20.0)) == (0.4, 0.0)
    assert tuple(o.dv1(25.0)) == (0.4, 0.0)
    assert tuple(o.dv1(10.0)) == (0.0, 0.0)
    assert tuple(o.dv1(3.0)) == (0.0, 0.0)
    # midpoint, m = 2: t = 1/2, [1 - t^2]^2 = 9/16
    assert o.dv1(15.0)[0] == pytest.approx(0.4 * 9.0 / 16.0, rel=1e-15)
    # continuous, C1 at both ends, monotone, within [0, dvmax] (Sec. 3.2.1 after Eq. 15)
    s = np.linspace(10.0, 20.0, 401)
    vals = np.array([o.dv1(v) for v in s])
    assert np.all(np.diff(vals[:, 0]) >= 0) and vals[:, 0].min() >= 0 and vals[:, 0].max() <= 0.4
    assert o.dv1(10.0 + 1e-7)[0] < 1e-12 and abs(o.dv1(20.0 - 1e-7)[0] - 0.4) < 1e-12
    assert abs(o.dv1(10.0 + 1e-6)[1]) < 1e-6 and abs(o.dv1(20.0 - 1e-6)[1]) < 1e-6
    h = 1e-6
    for v in (11.0, 13.3, 17.9):
        fd = (o.dv1(v + h)[0] - o.dv1(v - h)[0]) / (2 * h)
        assert fd == pytest.approx(o.dv1(v)[1], rel=1e-7)
    for m in (3, 4):
        r.m_exp = m
        o = oracle_mod.OracleReplica(r, _params(bias_on=1))
        t = 0.5
        assert o.dv1(15.0)[0] == pytest.approx(0.4 * (1 - t ** m) ** 2, rel=1e-15)


@pytest.mark.parametrize("mk", [small2d, small3d])
def test_bias_force_by_differences(oracle_mod, mk):
    base = mk()
    o0 = oracle_mod.OracleReplica(base, _params())
    xq, _, _ = o0.quench(method=1, ftol=1e-9, max_iter=20000)
    r = base.copy()
    r.pos_ref = xq
    r.pos = thermalise(base, amp=0.05, seed=5).pos - base.pos + xq
    probe = oracle_mod.OracleReplica(r, _params())
    s0 = probe.s.sigma
    r.dvmax, r.sig_lo, r.sig_hi, r.m_exp = 0.3, 0.5 * s0, 1.5 * s0, 2
    o = oracle_mod.OracleReplica(r, _params(bias_on=1))
    assert 0.0 < o.s.dV < 0.3                         # inside the interpolation region
    x = o.x.copy()
    h = 1e-5

    def vb(xx):
        return o.potential(xx) + o.bias_potential(xx)

    assert o.bias_potential(x) == pytest.approx(o.s.dV, rel=1e-12)
    for i in [k for k in range(r.n) if r.role[k] == 1][:: max(1, r.n // 20)]:
        for a in range(r.dim):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -(vb(xp) - vb(xm)) / (2 * h)
            assert fd == pytest.approx(o.ftot[i, a], rel=1e-6, abs=1e-6)
    rig = r.role == 2
    for a in range(r.dim):
        xp, xm = x.copy(), x.copy()
        xp[rig, a] += h
        xm[rig, a] -= h
        fd = -(vb(xp) - vb(xm)) / (2 * h)
        assert fd == pytest.approx(o.s.fbody[a], rel=1e-6, abs=1e-6)
    # d and sigma follow Eq. 7 and Eq. 5 from first principles
    dr = x - o.xo
    assert o.s.d == pytest.approx(np.sqrt((dr ** 2).sum()), rel=1e-13)
    assert o.s.sigma == pytest.approx((o.gradient() * dr).sum() / o.s.d, rel=1e-10)


# ---------------------------------------------------------------- dynamics
def _equilibrated(mk, steps=1500, **kw):
    from oracle import oracle as O
    base = mk(**kw)
    o = O.OracleReplica(base, _params())
    xq, _, _ = o.quench(method=1, ftol=1e-8, max_iter=20000)
    r = base.copy()
    r.pos, r.pos_ref = xq.copy(), xq.copy()
    o = O.OracleReplica(r, _params())
    o.run(steps)
    st = r.copy()
    st.pos, st.vel = o.x.copy(), o.v.copy()
    return st


@pytest.mark.parametrize("bias", [0, 1])
def test_nve_second_order(oracle_mod, bias):
    st = _equilibrated(small2d)
    drifts = []
    for dt in (0.005, 0.0025):
        s = st.copy()
        s.gamma = 0.0
        if bias:
            s.dvmax, s.sig_lo, s.sig_hi = 0.3, 10.0, 30.0
        o = oracle_mod.OracleReplica(s, _params(bias_on=bias, dt=dt))
        e0 = o.s.K + o.s.V + o.s.dV
        dev = 0.0
        nst = int(round(0.5 / dt))
        for _ in range(12):
            o.run(nst)
            dev = max(dev, abs(o.s.K + o.s.V + o.s.dV - e0))
        drifts.append(dev)
        assert dev < 5e-3 * (dt / 0.005) ** 2 * 10
    # velocity-Verlet family: energy error ~ dt^2
    assert 3.0 < drifts[0] / drifts[1] < 5.0


def test_boost_one_reduces_to_plain_md(oracle_mod):
    st = _equilibrated(small2d, steps=200)
    plain = oracle_mod.OracleReplica(st.copy(), _params(bias_on=0))
    s = st.copy()
    s.dvmax, s.sig_lo, s.sig_hi = 0.0, 1.0, 2.0
    zero = oracle_mod.OracleReplica(s, _params(bias_on=1))
    plain.run(300)
    zero.run(300)
    assert np.array_equal(plain.x, zero.x) and np.array_equal(plain.v, zero.v)
    assert zero.s.t_h == zero.s.t_md == plain.s.t_md
    assert zero.s.t_h == pytest.approx(300 * 0.005, rel=1e-13)


def test_saturated_bias_gives_constant_boost(oracle_mod):
    """sigma always above sigma_U: DeltaV = DeltaV_max is a constant, the force is
    unbiased and the clock runs exp(beta DeltaV_max) times faster (Eq. 3)."""
    st = _equilibrated(small2d, steps=200)
    plain = oracle_mod.OracleReplica(st.copy(), _params(bias_on=0))
    s = st.copy()
    s.dvmax, s.sig_lo, s.sig_hi = 0.25, -2.0, -1.0
    sat = oracle_mod.OracleReplica(s, _params(bias_on=1))
    plain.run(200)
    sat.run(200)
    assert np.array_equal(plain.x, sat.x)
    assert sat.s.t_h == pytest.approx(200 * 0.005 * np.exp(0.25 / s.kT), rel=1e-12)


@pytest.mark.parametrize("bias", [0, 1])
def test_equipartition(oracle_mod, bias):
    s = _equilibrated(small2d, steps=1000, kT=0.08)
    if bias:
        s.dvmax, s.sig_lo, s.sig_hi = 0.3, 8.0, 20.0
    o = oracle_mod.OracleReplica(s, _params(bias_on=bias))
    mob = s.role == 1
    acc, cnt = 0.0, 0
    for _ in range(150):
        o.run(100)
        acc += (o.v[mob][:, :2] ** 2).mean()
        cnt += 1
    assert acc / cnt == pytest.approx(0.08, rel=0.03)


# ---------------------------------------------------------------- quench and transitions
@pytest.mark.parametrize("mk", [small2d, small3d])
def test_quench_returns_to_minimum(oracle_mod, mk):
    """Both minimisers bring a slightly displaced minimum back to it.  Positions
    agree within ftol / (softest stiffness).  The cutoff shifts energies but not
    forces, so pairs near rc put kinks in the 3-D landscape with stationary
    points 1e-4 apart in energy; there the energy check is loose."""
    base = mk()
    o = oracle_mod.OracleReplica(base, _params())
    xstar, _, fm = o.quench(method=1, ftol=1e-9, max_iter=40000)
    assert fm < 1e-9
    r = base.copy()
    r.pos = thermalise(base, amp=0.01 if base.dim == 2 else 0.002, seed=9).pos - base.pos + xstar
    o2 = oracle_mod.OracleReplica(r, _params())
    xs, its, fs = o2.quench(method=0, ftol=1e-6, max_iter=100000, step_size=0.002)
    xf, itf, ff = o2.quench(method=1, ftol=1e-6, max_iter=100000)
    assert fs < 1e-6 and ff < 1e-6
    tol = 1e-5 if base.dim == 2 else 3e-3
    assert np.abs(xs - xstar).max() < tol and np.abs(xf - xstar).max() < tol
    e0 = o2.potential(xstar)
    etol = 1e-9 if base.dim == 2 else 1e-4
    assert abs(o2.potential(xs) - e0) < etol and abs(o2.potential(xf) - e0) < etol
    assert itf < its                                     # FIRE needs fewer steps than SD
    assert np.array_equal(o2.x, r.pos)                  # the quench leaves the MD state alone


def test_transition_flag(oracle_mod):
    base = small2d()
    o = oracle_mod.OracleReplica(base, _params())
    xstar, _, _ = o.quench(method=1, ftol=1e-8, max_iter=40000)
    ref = base.copy()
    ref.pos, ref.pos_ref = xstar.copy(), xstar.copy()
    # unperturbed thermal state: quench comes back to r_O
    st = ref.copy()
    st.pos = thermalise(ref, amp=0.03, seed=2).pos
    o1 = oracle_mod.OracleReplica(st, _params())
    xq, _, _ = o1.quench(method=1, ftol=1e-6, max_iter=40000)
    flag, md = o1.transition(xq, 0.5)
    assert not flag and md < 0.05
    # forced slip: the whole tip moved by one lattice spacing along x
    sl = ref.copy()
    sl.pos = xstar.copy()
    sl.pos[sl.type == 1, 0] += 2.0 ** (1.0 / 6.0)
    o2 = oracle_mod.OracleReplica(sl, _params())
    xq2, _, _ = o2.quench(method=1, ftol=1e-6, max_iter=40000)
    flag2, md2 = o2.transition(xq2, 0.5)
    assert flag2 and md2 > 0.9


def _maxdisp(r, x):
    """Largest minimum-image displacement of x from the replica's r_O (numpy)."""
    d = x - r.pos_ref
    for a in range(3):
        if r.periodic[a]:
            d[:, a] -= r.box[a] * np.rint(d[:, a] / r.box[a])
    return float(np.sqrt((d * d).sum(axis=1)).max())


def test_gated_quench_gives_the_full_quench_answer(oracle_mod):
    """The quench that stops early in its basin (max|F| < ftol_stay with every
    atom within keep = theta/2 of r_O) gives the transition test the answer of
    the quench run to ftol: on a thermal state it stops sooner, within
    theta - keep of the full quench's minimum, unflagged; on a forced slip the
    early stop never applies and the two quenches are identical; with
    ftol_stay = 0 it is the plain quench."""
    base = small2d()
    o = oracle_mod.OracleReplica(base, _params())
    xstar, _, _ = o.quench(method=1, ftol=1e-8, max_iter=40000)
    ref = base.copy()
    ref.pos, ref.pos_ref = xstar.copy(), xstar.copy()
    theta, keep = 0.5, 0.25
    st = ref.copy()
    st.pos = thermalise(ref, amp=0.03, seed=2).pos
    o1 = oracle_mod.OracleReplica(st, _params())
    xf, itf, ff = o1.quench(method=1, ftol=1e-6, max_iter=40000, step_size=0.005)
    xg, itg, fg = o1.quench(method=1, ftol=1e-6, max_iter=40000, step_size=0.005, ftol_stay=1e-1, keep=keep)
    assert ff < 1e-6 and 1e-6 <= fg < 1e-1
    assert itg < itf
    assert _maxdisp(st, xg) < keep and _maxdisp(st, xf) < theta
    assert np.abs(xg - xf).max() < theta - keep
    assert o1.transition(xg, theta)[0] == o1.transition(xf, theta)[0] == 0
    x0, it0, f0 = o1.quench(method=1, ftol=1e-6, max_iter=40000, step_size=0.005, ftol_stay=0.0, keep=keep)
    assert np.array_equal(x0, xf) and it0 == itf and f0 == ff
    sl = ref.copy()
    sl.pos = xstar.copy()
    sl.pos[sl.type == 1, 0] += 2.0 ** (1.0 / 6.0)
    o2 = oracle_mod.OracleReplica(sl, _params())
    xf2, itf2, _ = o2.quench(method=1, ftol=1e-6, max_iter=40000, step_size=0.005)
    xg2, itg2, _ = o2.quench(method=1, ftol=1e-6, max_iter=40000, step_size=0.005, ftol_stay=1e-1, keep=keep)
    assert itg2 == itf2 and np.array_equal(xg2, xf2)
    assert o2.transition(xg2, theta)[0] == 1 and _maxdisp(sl, xg2) > 0.9


def test_gated_quench_on_a_3d_model(oracle_mod):
    """3-D: from a thermal state around the minimum the in-basin stop comes
    sooner, within theta - keep of the full quench's minimum and unflagged;
    against an r_O moved by 0.6 sigma it never applies (the quench equals the
    full one, flagged)."""
    base = small3d()
    o = oracle_mod.OracleReplica(base, _params())
    xstar, _, _ = o.quench(method=1, ftol=1e-8, max_iter=40000)
    ref = base.copy()
    ref.pos, ref.pos_ref = xstar.copy(), xstar.copy()
    theta, keep = 0.5, 0.25
    st = ref.copy()
    st.pos = thermalise(ref, amp=0.02, seed=5).pos
    o1 = oracle_mod.OracleReplica(st, _params())
    xf, itf, ff = o1.quench(method=1, ftol=1e-4, max_iter=40000, step_size=0.005)
    xg, itg, fg = o1.quench(method=1, ftol=1e-4, max_iter=40000, step_size=0.005, ftol_stay=1e-1, keep=keep)
    assert ff < 1e-4 and fg < 1e-1 and itg < itf
    assert _maxdisp(st, xg) < keep and np.abs(xg - xf).max() < theta - keep
    assert o1.transition(xg, theta)[0] == o1.transition(xf, theta)[0] == 0
    far = st.copy()
    far.pos_ref = st.pos_ref.copy()
    far.pos_ref[:, 0] += 0.6
    o2 = oracle_mod.OracleReplica(far, _params())
    xf2, itf2, _ = o2.quench(method=1, ftol=1e-4, max_iter=40000, step_size=0.005)
    xg2, itg2, _ = o2.quench(method=1, ftol=1e-4, max_iter=40000, step_size=0.005, ftol_stay=1e-1, keep=keep)
    assert itg2 == itf2 and np.array_equal(xg2, xf2)
    assert o2.transition(xg2, theta)[0] == 1


def test_diverging_quench_stops_cleanly(oracle_mod):
    """Steepest descent with a step beyond 2 / (largest curvature) runs away
    from a thermal configuration of the paper's 2-D model: the quench must
    stop early with fmax = NaN, not build a cell grid from runaway
    coordinates, and leave the MD state alone."""
    from paper_0909_5215_gb300 import model as M
    base = M.paper2d(kT=0.01)
    st = thermalise(base, amp=0.05, seed=4)
    o = oracle_mod.OracleReplica(st, _params())
    x0 = o.x.copy()
    xq, it, fm = o.quench(method=0, ftol=1e-4, max_iter=2000, step_size=0.05)
    assert np.isnan(fm) and it < 2000
    assert np.array_equal(o.x, x0)
    # the same state with a stable step converges
    xq, it, fm = o.quench(method=0, ftol=1e-4, max_iter=200000, step_size=0.002)
    assert fm < 1e-4
