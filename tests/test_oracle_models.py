"""The paper's own models (Sec. 3.1.1, Sec. 3.2.1) and the harmonic tip bonds
of Eq. 12 in the oracle.

* Preset sizes, roles and parameters as the paper states them, the 3-D tip's
  contact layer of nine atoms in registry with the substrate, and bonds at the
  nearest-neighbour distance.
* Eq. 12 in closed form and its stiffness against the LJ curvature at its
  minimum (the paper picks k and r_O to match it).
* With bonds, the total potential equals a direct sum written out here (LJ for
  every pair but tip-tip, bonds, spring and load), the list forces equal an
  all-pairs sum, forces and H.dr equal finite differences, the eigenvalue
  gradient equals finite differences of the eigenvalue, and NVE energy error
  falls as dt^2.
"""
import numpy as np
import pytest

from conftest import small3d, thermalise


def _params(**kw):
    from paper_0909_5215_gb300 import model as M
    return M.Params(**kw)


def test_paper_2d_model():
    from paper_0909_5215_gb300 import model as M
    r = M.paper2d()
    assert ((r.type == 0).sum(), (r.type == 1).sum()) == (80, 33)
    assert ((r.role == 0).sum(), (r.role == 2).sum()) == (20, 8)
    assert (r.k_spring, r.f_normal) == (5.0, 5.0) and r.eps == M.PAPER_EPS_2D
    # tip rows of 3, 4, ..., 8 atoms; neighbours in the tip at the lattice spacing
    y = np.round(r.pos[r.type == 1, 1], 6)
    assert sorted(np.unique(y, return_counts=True)[1]) == [3, 4, 5, 6, 7, 8]
    t = r.pos[r.type == 1]
    d = np.sqrt(((t[:, None] - t[None]) ** 2).sum(-1)) + np.eye(len(t)) * 9
    assert np.allclose(d.min(1), M.A2D)


def test_paper_3d_model():
    from paper_0909_5215_gb300 import model as M
    r = M.paper3d()
    assert ((r.type == 0).sum(), (r.type == 1).sum()) == (1800, 183)
    assert ((r.role == 0).sum(), (r.role == 2).sum()) == (450, 60)
    assert (r.k_spring, r.f_normal) == (10.0, 5.0) and r.eps == M.PAPER_EPS_3D
    tip = r.pos[r.type == 1]
    z, cnt = np.unique(np.round(tip[:, 2], 6), return_counts=True)
    assert list(cnt) == [9, 16, 21, 32, 45, 60]
    # contact layer on the fcc sites one half cell above the substrate: every
    # contact atom sits over the centre of four top-layer substrate atoms
    sub = r.pos[r.type == 0]
    top = sub[np.isclose(sub[:, 2], sub[:, 2].max())]
    assert z[0] == pytest.approx(sub[:, 2].max() + M.AFCC / 2)
    for p in tip[np.isclose(tip[:, 2], z[0])]:
        dxy = top[:, :2] - p[:2]
        dxy -= r.box[:2] * np.rint(dxy / r.box[:2])
        assert (np.sqrt((dxy ** 2).sum(1)) < M.AFCC / np.sqrt(2) / 2 + 1e-6).sum() == 0
        assert np.isclose(np.sqrt((dxy ** 2).sum(1)), M.AFCC / 2).sum() == 4
    # bonds join tip atoms at the nearest-neighbour distance; bulk atoms have 12
    b = r.bonds
    assert np.all(r.type[b] == 1)
    L = np.linalg.norm(r.pos[b[:, 0]] - r.pos[b[:, 1]], axis=1)
    assert np.allclose(L, M.AFCC / np.sqrt(2))
    assert np.bincount(b.ravel(), minlength=r.n).max() == 12


def test_eq12_matches_lj_minimum(oracle_mod):
    """k = 57.2 and r_O = 1.12 are the LJ curvature 72 / 2^(1/3) = 57.146 and
    minimum 2^(1/6) = 1.1225, to the digits printed."""
    assert 57.2 == pytest.approx(72.0 / 2.0 ** (1.0 / 3.0), abs=0.06)
    assert 1.12 == pytest.approx(2.0 ** (1.0 / 6.0), abs=0.003)


def _bonded_small(amp=0.05, seed=3):
    from paper_0909_5215_gb300 import model as M
    r = thermalise(small3d(nx=5, nz=3, radius=3.0), amp=amp, seed=seed)
    r.bonds = M.tip_bonds(small3d(nx=5, nz=3, radius=3.0))
    r.pos_ref = small3d(nx=5, nz=3, radius=3.0).pos.copy()
    return r


def _direct_potential(r, x, rc=2.5):
    """LJ over every pair closer than rc except tip-tip ones, shifted to zero
    at rc (Eq. 9); Eq. 12 over the bonds; spring and load on the rigid layer."""
    def lj(q, e):
        return 4 * e * (q ** -12 - q ** -6)
    n = r.n
    d = x[:, None, :] - x[None, :, :]
    for a in range(3):
        if r.periodic[a]:
            d[..., a] -= r.box[a] * np.rint(d[..., a] / r.box[a])
    q = np.sqrt((d ** 2).sum(-1))
    v = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            if q[i, j] < rc and not (r.type[i] == 1 and r.type[j] == 1):
                e = r.eps[r.type[i]][r.type[j]]
                v += lj(q[i, j], e) - lj(rc, e)
    for i, j in r.bonds:
        v += 0.5 * r.k_bond * (q[i, j] - r.r_bond) ** 2
    rig = r.role == 2
    xt = x[rig].mean(0)
    v += 0.5 * r.k_spring * ((xt[0] - r.slider[0]) ** 2 + (xt[1] - r.slider[1]) ** 2) + r.f_normal * xt[2]
    return v


def test_bonded_potential_is_the_direct_sum(oracle_mod):
    r = _bonded_small()
    o = oracle_mod.OracleReplica(r, _params())
    assert o.potential() == pytest.approx(_direct_potential(r, r.pos), rel=1e-12)


def test_bonded_forces_list_brute_and_gradient(oracle_mod):
    r = _bonded_small()
    o = oracle_mod.OracleReplica(r, _params())
    o.nlist_cells()
    o.forces()
    fb, _, vb = o.forces_brute()
    assert np.sqrt(((o.f_lj - fb) ** 2).sum() / (fb ** 2).sum()) < 1e-13
    rng = np.random.default_rng(4)
    h = 1e-5
    for _ in range(3):
        u = rng.normal(size=(r.n, 3))
        u[r.role == 0] = 0.0
        u[r.role == 2] = u[r.role == 2][0]
        u /= np.linalg.norm(u)
        fd = (o.potential(o.x + h * u) - o.potential(o.x - h * u)) / (2 * h)
        assert np.sum(o.gradient() * u) == pytest.approx(fd, rel=1e-6)


def test_bonded_hessian_vector(oracle_mod):
    r = _bonded_small()
    o = oracle_mod.OracleReplica(r, _params())
    rng = np.random.default_rng(5)
    u = rng.normal(size=(r.n, 3))
    u /= np.linalg.norm(u)
    h = 1e-5
    fd = (o.gradient(o.x + h * u) - o.gradient(o.x - h * u)) / (2 * h)
    hv = o.hessvec(u)
    assert np.sqrt(((hv - fd) ** 2).sum() / (fd ** 2).sum()) < 1e-7
    # and the H.dr the force routine returns with the list
    o.nlist_cells()
    o.forces()
    dr = o.x - o.xo
    hd = o.hessvec(dr)
    rig = r.role == 2
    assert np.allclose(o.hdr[~rig], hd[~rig], rtol=1e-10, atol=1e-10)


def test_bonded_eigenvalue_gradient(oracle_mod):
    r = _bonded_small(seed=9)
    o = oracle_mod.OracleReplica(r, _params())
    e, v = o.lowest_eig()
    g = o.eig_grad(v)
    rng = np.random.default_rng(6)
    h = 1e-5
    for _ in range(2):
        u = o.project(rng.normal(size=(r.n, 3)))
        u /= np.linalg.norm(u)
        ep, _ = o.lowest_eig(x=o.x + h * u, v0=v)
        em, _ = o.lowest_eig(x=o.x - h * u, v0=v)
        assert (ep - em) / (2 * h) == pytest.approx(np.sum(g * u), rel=2e-6, abs=1e-6)


def test_bonded_nve_second_order(oracle_mod):
    """The paper's 2-D model with its tip held by Eq. 12 bonds: NVE energy error
    ~ dt^2.  (In 3-D the many pairs crossing the cutoff, where the shifted LJ
    force jumps, add an error of first order that masks the dt^2 law, with or
    without bonds.)"""
    from paper_0909_5215_gb300 import model as M
    base = M.paper2d()
    base.bonds = M.tip_bonds(base)
    o = oracle_mod.OracleReplica(base, _params())
    xq, _, _ = o.quench(method=1, ftol=1e-8, max_iter=20000)
    r = base.copy()
    r.pos, r.pos_ref = xq.copy(), xq.copy()
    o = oracle_mod.OracleReplica(r, _params())
    o.run(1000)
    st = r.copy()
    st.pos, st.vel = o.x.copy(), o.v.copy()
    devs = []
    for dt in (0.004, 0.002):
        s = st.copy()
        s.gamma = 0.0
        o = oracle_mod.OracleReplica(s, _params(dt=dt))
        e0, dev = o.s.K + o.s.V, 0.0
        for _ in range(5):
            o.run(int(round(0.1 / dt)))
            dev = max(dev, abs(o.s.K + o.s.V - e0))
        devs.append(dev)
    assert devs[0] < 5e-3
    assert 3.0 < devs[0] / devs[1] < 5.0
