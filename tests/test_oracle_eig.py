"""Pins of the oracle's eigenvalue bias (Eq. 13, Eq. 15) to things other than itself.

epsilon is the lowest eigenvalue of the Hessian over the allowed motions
(fixed atoms frozen, rigid layer as one body, 3N metric).  Pinned here:
  * phi''' of the LJ pair against its closed form at the minimum and a
    finite difference of phi'';
  * a dimer (one fixed, one mobile atom): epsilon = min(phi'(r)/r, phi''(r)),
    the transverse and the bond curvature, and grad epsilon = (B r) or phi''';
  * Lanczos against a dense symmetric eigensolver on the reduced Hessian
    Q^T H Q of small 2-D and 3-D models (Q an orthonormal basis of the
    allowed motions);
  * grad epsilon against central differences of epsilon itself;
  * Eq. 15 breakpoints and derivative, Eq. 13 reductions and range;
  * the total force with both terms active against finite differences of
    V + DeltaV, and NVE conservation of K + V + DeltaV with error ~ dt^2.
"""
import numpy as np
import pytest

from conftest import small2d, small3d, thermalise


def _params(**kw):
    from paper_0909_5215_gb300 import model as M
    return M.Params(**kw)


def _dimer(rho, dim):
    from paper_0909_5215_gb300 import model as M
    return M.Replica(dim=dim, pos=np.array([[0.0, 0.0, 0.0], [rho, 0.0, 0.0]]),
                     role=np.array([0, 1], np.uint8), type=np.zeros(2, np.uint8),
                     box=np.zeros(3), periodic=np.zeros(3, np.uint8), kT=0.1, k_spring=0.0, f_normal=0.0,
                     slider=np.zeros(2), eps=((1.0, 1.0), (1.0, 1.0)))


def _phi(oracle_mod, r):
    out = np.zeros(3)
    oracle_mod.lib().or_lj(r, 1.0, 1.0, 2.5, out.ctypes.data_as(oracle_mod.C.POINTER(oracle_mod.C.c_double)))
    return out


def test_lj_third_derivative(oracle_mod):
    r0 = 2.0 ** (1.0 / 6.0)
    # at the minimum (sigma/r)^6 = 1/2: phi''' = 4 (-2184/4 + 336/2) / r0^3 = -1512 / sqrt(2)
    assert oracle_mod.lib().or_lj3(r0, 1.0, 1.0) == pytest.approx(-1512.0 / np.sqrt(2.0), rel=1e-13)
    for r in (0.95, 1.1, 1.4, 2.0):
        h = 1e-5
        fd = (_phi(oracle_mod, r + h)[2] - _phi(oracle_mod, r - h)[2]) / (2 * h)
        assert oracle_mod.lib().or_lj3(r, 1.0, 1.0) == pytest.approx(fd, rel=1e-7)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("rho", [0.97, 1.05, 2.0 ** (1.0 / 6.0), 1.2, 1.3, 1.7])
def test_dimer_closed_form(oracle_mod, dim, rho):
    o = oracle_mod.OracleReplica(_dimer(rho, dim), _params())
    e, v = o.lowest_eig()
    ph = _phi(oracle_mod, rho)
    transverse, bond = ph[1] / rho, ph[2]
    assert e == pytest.approx(min(transverse, bond), rel=1e-10, abs=1e-10)
    g = o.eig_grad(v)
    if bond < transverse - 1e-9:
        assert abs(v[1, 0]) == pytest.approx(1.0, rel=1e-10)
        want = oracle_mod.lib().or_lj3(rho, 1.0, 1.0)             # d phi''/d rho
    elif transverse < bond - 1e-9:
        assert abs(v[1, 0]) < 1e-8
        want = (bond - transverse) / rho                          # d (phi'/rho)/d rho = B rho
    else:
        return                                                    # degenerate at the minimum
    assert g[1, 0] == pytest.approx(want, rel=1e-10)
    assert np.allclose(g[1, 1:], 0.0, atol=1e-10) and np.allclose(g[0], -g[1])


def _allowed_basis(r):
    """Orthonormal basis of the allowed motions: mobile coordinates and the
    rigid body's translation (1/sqrt(n_rig) on every rigid atom)."""
    n, cols = r.n, []
    rig = np.nonzero(r.role == 2)[0]
    for i in np.nonzero(r.role == 1)[0]:
        for a in range(r.dim):
            q = np.zeros((n, 3))
            q[i, a] = 1.0
            cols.append(q)
    for a in range(r.dim if rig.size else 0):
        q = np.zeros((n, 3))
        q[rig, a] = 1.0 / np.sqrt(rig.size)
        cols.append(q)
    return cols


@pytest.mark.parametrize("mk", [small2d, small3d])
def test_lanczos_equals_dense_eigensolver(oracle_mod, mk):
    r = thermalise(mk(), amp=0.06, seed=5)
    o = oracle_mod.OracleReplica(r, _params())
    Q = _allowed_basis(r)
    HQ = [o.hessvec(q) for q in Q]
    Hr = np.array([[np.sum(qa * hb) for hb in HQ] for qa in Q])
    assert np.allclose(Hr, Hr.T, atol=1e-9)
    w, y = np.linalg.eigh(0.5 * (Hr + Hr.T))
    e, v = o.lowest_eig()
    assert e == pytest.approx(w[0], rel=1e-9, abs=1e-9)
    vd = sum(c * q for c, q in zip(y[:, 0], Q))
    assert abs(np.sum(v * vd)) == pytest.approx(1.0, abs=1e-7)
    assert np.allclose(o.project(v), v)                           # v is an allowed motion


@pytest.mark.parametrize("mk", [small2d, small3d])
def test_eigenvalue_gradient_is_its_derivative(oracle_mod, mk):
    r = thermalise(mk(), amp=0.06, seed=7)
    o = oracle_mod.OracleReplica(r, _params())
    e, v = o.lowest_eig()
    g = o.eig_grad(v)
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(3):
        u = o.project(rng.normal(size=(r.n, 3)))
        u /= np.linalg.norm(u)
        ep, _ = o.lowest_eig(x=o.x + h * u, v0=v)
        em, _ = o.lowest_eig(x=o.x - h * u, v0=v)
        fd = (ep - em) / (2 * h)
        assert fd == pytest.approx(np.sum(g * u), rel=2e-6, abs=1e-6)


def test_eq15_and_eq13(oracle_mod):
    r = small2d()
    r.dvmax, r.m_exp, r.eig_lo, r.eig_hi = 0.3, 2, -0.5, 1.5
    o = oracle_mod.OracleReplica(r, _params())
    assert tuple(o.dv2(1.5)) == (0.3, 0.0) and tuple(o.dv2(2.0)) == (0.3, 0.0)
    assert tuple(o.dv2(-0.5)) == (0.0, 0.0) and tuple(o.dv2(-1.0)) == (0.0, 0.0)
    for e in (-0.3, 0.2, 0.9, 1.4):
        h = 1e-6
        assert o.dv2(e)[1] == pytest.approx((o.dv2(e + h)[0] - o.dv2(e - h)[0]) / (2 * h), rel=1e-6)
    assert o.dv2(1.5 - 1e-7)[0] == pytest.approx(0.3, rel=1e-9)       # continuous at both ends
    assert o.dv2(-0.5 + 1e-7)[0] == pytest.approx(0.0, abs=1e-12)
    g = np.linspace(0.0, 0.3, 7)
    for a in g:
        assert o.dv13(a, 0.0)[0] == pytest.approx(a) and o.dv13(0.0, a)[0] == pytest.approx(a)
        assert o.dv13(a, 0.3)[0] == pytest.approx(0.3) and o.dv13(0.3, a)[0] == pytest.approx(0.3)
        for b in g:
            c = o.dv13(a, b)
            assert -1e-15 <= c[0] <= 0.3 + 1e-15
            assert c[0] == pytest.approx(o.dv13(b, a)[0])
            assert c[1] == pytest.approx(1.0 - b / 0.3) and c[2] == pytest.approx(1.0 - a / 0.3)


def _both_active(oracle_mod, mk, seed):
    """An equilibrated model (quench, then Langevin MD) with sigma and
    epsilon both inside their bands."""
    base = mk()
    o = oracle_mod.OracleReplica(base, _params())
    xq, _, _ = o.quench(method=1, ftol=1e-8, max_iter=20000)
    r = base.copy()
    r.pos, r.pos_ref, r.rep_id = xq.copy(), xq.copy(), seed
    o = oracle_mod.OracleReplica(r, _params())
    o.run(1000)
    r.pos, r.vel = o.x.copy(), o.v.copy()
    o = oracle_mod.OracleReplica(r, _params(bias_on=1))
    s0 = o.s.sigma
    e0, _ = o.lowest_eig()
    r.dvmax, r.m_exp, r.eig_on = 0.3, 2, 1
    r.sig_lo, r.sig_hi = s0 - 0.5 * abs(s0) - 0.1, s0 + 0.5 * abs(s0) + 0.1
    r.eig_lo, r.eig_hi = e0 - 0.5 * abs(e0) - 0.05, e0 + 0.5 * abs(e0) + 0.05
    return r


@pytest.mark.parametrize("mk", [small2d, small3d])
def test_combined_bias_force_is_minus_gradient(oracle_mod, mk):
    r = _both_active(oracle_mod, mk, seed=11)
    p = _params(bias_on=1)
    o = oracle_mod.OracleReplica(r, p)
    assert 0.0 < o.s.dV1 < 0.3 and 0.0 < o.s.dV2 < 0.3 and o.s.dVe != 0.0
    assert o.s.dV == pytest.approx(o.s.dV1 + o.s.dV2 - o.s.dV1 * o.s.dV2 / 0.3, rel=1e-13)
    ft = o.ftot.copy()
    rng = np.random.default_rng(2)
    h = 1e-5
    for _ in range(3):
        u = o.project(rng.normal(size=(r.n, 3)))
        u /= np.linalg.norm(u)
        ep = o.potential(o.x + h * u) + o.bias_potential(o.x + h * u)
        em = o.potential(o.x - h * u) + o.bias_potential(o.x - h * u)
        fd = (ep - em) / (2 * h)
        assert -np.sum(ft * u) == pytest.approx(fd, rel=1e-5, abs=1e-6)


def test_nve_with_eigenvalue_bias_second_order(oracle_mod):
    """K + V + DeltaV conserved with an error ~ dt^2 while the lowest
    eigenvalue stays simple (epsilon is not differentiable where two
    eigenvalues cross, and a crossing breaks the dt^2 law); this state's two
    lowest eigenvalues are about 1 apart."""
    r = _both_active(oracle_mod, small2d, seed=17)
    drifts = []
    for dt in (0.002, 0.001):
        s = r.copy()
        s.gamma = 0.0
        o = oracle_mod.OracleReplica(s, _params(bias_on=1, dt=dt))
        assert o.s.dVe != 0.0
        e0 = o.s.K + o.s.V + o.s.dV
        dev = 0.0
        for _ in range(5):
            o.run(int(round(0.01 / dt)))
            dev = max(dev, abs(o.s.K + o.s.V + o.s.dV - e0))
        drifts.append(dev)
    assert drifts[0] < 1e-3
    assert 3.0 < drifts[0] / drifts[1] < 5.0                      # velocity Verlet: error ~ dt^2
