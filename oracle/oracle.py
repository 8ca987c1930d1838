"""ctypes binding of the plain CPU FP64 oracle (hd_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference leg.  The product path never imports it.

`build()` compiles hd_oracle.c with gcc (-O2 -ffp-contract=off -fopenmp) into
liboracle.so beside this file.  `OracleReplica` holds one replica's numpy
arrays and the C struct that points at them.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hd_oracle.c")
_HDR = os.path.join(_HERE, "hd_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library if missing or older than its sources."""
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-std=c11", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrRep(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n", C.c_int), ("rep_id", C.c_int), ("m_exp", C.c_int),
        ("L", C.c_double * 3), ("periodic", C.c_int * 3),
        ("kT", C.c_double), ("gamma", C.c_double), ("kspring", C.c_double),
        ("fnormal", C.c_double), ("slider", C.c_double * 2),
        ("dvmax", C.c_double), ("sig_lo", C.c_double), ("sig_hi", C.c_double),
        ("eps", (C.c_double * 2) * 2), ("sig", (C.c_double * 2) * 2),
        ("x", C.POINTER(C.c_double)), ("v", C.POINTER(C.c_double)), ("xo", C.POINTER(C.c_double)),
        ("role", C.POINTER(C.c_uint8)), ("type", C.POINTER(C.c_uint8)),
        ("maxnb", C.c_int),
        ("nnb", C.POINTER(C.c_int)), ("nbr", C.POINTER(C.c_int)),
        ("xb", C.POINTER(C.c_double)),
        ("f_lj", C.POINTER(C.c_double)), ("hdr", C.POINTER(C.c_double)),
        ("e_atom", C.POINTER(C.c_double)), ("ftot", C.POINTER(C.c_double)),
        ("t_h", C.c_double), ("t_md", C.c_double),
        ("step", C.c_int64), ("n_rebuild", C.c_int64), ("nb_overflow", C.c_int64),
        ("vbody", C.c_double * 3),
        ("V", C.c_double), ("V_lj", C.c_double), ("K", C.c_double), ("dV", C.c_double),
        ("dVp", C.c_double), ("sigma", C.c_double), ("d", C.c_double), ("G", C.c_double),
        ("xT", C.c_double * 3), ("fbody", C.c_double * 3), ("FR", C.c_double),
        ("eig_on", C.c_int), ("eig_maxit", C.c_int), ("eig_lo", C.c_double), ("eig_hi", C.c_double),
        ("veig", C.POINTER(C.c_double)),
        ("eig", C.c_double), ("dV1", C.c_double), ("dV2", C.c_double), ("dVe", C.c_double),
        ("vslide", C.c_double), ("slide_x0", C.c_double), ("slide_step0", C.c_int64),
        ("nbond", C.c_int), ("bonds", C.POINTER(C.c_int)), ("kbond", C.c_double), ("rbond", C.c_double),
        ("nhc_len", C.c_int), ("nhc_tau", C.c_double), ("nhc_xi", C.c_double * 8), ("nhc_v", C.c_double * 8),
    ]


class OrParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("rc", C.c_double), ("skin", C.c_double),
                ("bias_on", C.c_int), ("seed", C.c_uint64)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        rp, pp = C.POINTER(OrRep), C.POINTER(OrParams)
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.or_unif.argtypes = [C.c_uint32, C.c_uint32]
        L.or_unif.restype = C.c_double
        L.or_normals.argtypes = [C.c_uint64, C.c_int, C.c_int64, C.c_int, C.c_int, dp]
        L.or_lj.argtypes = [C.c_double] * 4 + [dp]
        L.or_dv1.argtypes = [rp, C.c_double, dp]
        L.or_nlist_brute.argtypes = [rp, C.c_double]
        L.or_nlist_cells.argtypes = [rp, C.c_double]
        L.or_forces.argtypes = [rp, pp]
        L.or_forces.restype = C.c_double
        L.or_forces_brute.argtypes = [rp, pp, dp, dp]
        L.or_forces_brute.restype = C.c_double
        L.or_potential.argtypes = [rp, pp, dp]
        L.or_potential.restype = C.c_double
        L.or_gradient.argtypes = [rp, pp, dp, dp]
        L.or_hessvec.argtypes = [rp, pp, dp, dp, dp]
        L.or_bias_potential.argtypes = [rp, pp, dp]
        L.or_bias_potential.restype = C.c_double
        L.or_bias_eval.argtypes = [rp, pp]
        L.or_init.argtypes = [rp, pp, C.c_int]
        L.or_run.argtypes = [rp, pp, C.c_int]
        L.or_run_batch.argtypes = [rp, C.c_int, pp, C.c_int]
        L.or_quench.argtypes = [rp, pp, C.c_int, C.c_double, C.c_int, C.c_double, dp, dp]
        L.or_quench.restype = C.c_int
        L.or_quench_batch.argtypes = [rp, C.c_int, pp, C.c_int, C.c_double, C.c_int, C.c_double,
                                      C.POINTER(dp), dp, ip]
        L.or_quench_gated.argtypes = [rp, pp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                                      dp, dp]
        L.or_quench_gated.restype = C.c_int
        L.or_quench_batch_gated.argtypes = [rp, C.c_int, pp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                                            C.c_double, C.POINTER(dp), dp, ip]
        L.or_transition.argtypes = [rp, dp, C.c_double, dp]
        L.or_transition.restype = C.c_int
        L.or_num_threads.restype = C.c_int
        L.or_lj3.argtypes = [C.c_double] * 3
        L.or_lj3.restype = C.c_double
        L.or_project.argtypes = [rp, dp]
        L.or_lowest_eig.argtypes = [rp, pp, dp, dp, C.c_int, C.c_double]
        L.or_lowest_eig.restype = C.c_double
        L.or_eig_grad.argtypes = [rp, pp, dp, dp, dp]
        L.or_dv2.argtypes = [rp, C.c_double, dp]
        L.or_dv13.argtypes = [rp, C.c_double, C.c_double, dp]
        L.or_nhc_energy.argtypes = [rp]
        L.or_nhc_energy.restype = C.c_double
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(params) -> OrParams:
    return OrParams(params.dt, params.rc, params.skin, int(params.bias_on), int(params.seed))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals(seed, rep_id, step, atom, call):
    out = np.zeros(2)
    lib().or_normals(int(seed), int(rep_id), int(step), int(atom), int(call), _dp(out))
    return out


def lj(r, eps=1.0, sig=1.0, rc=2.5):
    out = np.zeros(3)
    lib().or_lj(float(r), float(eps), float(sig), float(rc), _dp(out))
    return out


class OracleReplica:
    """One replica in the oracle: numpy arrays plus the C struct over them."""

    def __init__(self, rep, params, maxnb: int | None = None, draw_velocities: bool | None = None):
        n = rep.n
        self.params = params
        self.P = make_params(params)
        self.maxnb = maxnb or (48 if rep.dim == 2 else 160)
        self.x = np.ascontiguousarray(rep.pos, dtype=np.float64).copy()
        self.v = (np.zeros((n, 3)) if rep.vel is None else np.ascontiguousarray(rep.vel, dtype=np.float64).copy())
        self.xo = (self.x.copy() if rep.pos_ref is None else np.ascontiguousarray(rep.pos_ref, dtype=np.float64).copy())
        self.role = np.ascontiguousarray(rep.role, dtype=np.uint8)
        self.type = np.ascontiguousarray(rep.type, dtype=np.uint8)
        self.nnb = np.zeros(n, dtype=np.int32)
        self.nbr = np.full((n, self.maxnb), -1, dtype=np.int32)
        self.xb = self.x.copy()
        self.f_lj = np.zeros((n, 3))
        self.hdr = np.zeros((n, 3))
        self.e_atom = np.zeros(n)
        self.ftot = np.zeros((n, 3))
        s = OrRep()
        s.dim, s.n, s.rep_id, s.m_exp = rep.dim, n, int(rep.rep_id), int(rep.m_exp)
        for a in range(3):
            s.L[a] = float(rep.box[a])
            s.periodic[a] = int(rep.periodic[a])
        s.kT, s.gamma, s.kspring, s.fnormal = rep.kT, rep.gamma, rep.k_spring, rep.f_normal
        s.slider[0], s.slider[1] = float(rep.slider[0]), float(rep.slider[1])
        s.dvmax, s.sig_lo, s.sig_hi = rep.dvmax, rep.sig_lo, rep.sig_hi
        for a in range(2):
            for b in range(2):
                s.eps[a][b] = float(rep.eps[a][b])
                s.sig[a][b] = float(rep.sig[a][b])
        s.x, s.v, s.xo = _dp(self.x), _dp(self.v), _dp(self.xo)
        s.role = self.role.ctypes.data_as(C.POINTER(C.c_uint8))
        s.type = self.type.ctypes.data_as(C.POINTER(C.c_uint8))
        s.maxnb = self.maxnb
        s.nnb = self.nnb.ctypes.data_as(C.POINTER(C.c_int))
        s.nbr = self.nbr.ctypes.data_as(C.POINTER(C.c_int))
        s.xb = _dp(self.xb)
        s.f_lj, s.hdr, s.e_atom, s.ftot = _dp(self.f_lj), _dp(self.hdr), _dp(self.e_atom), _dp(self.ftot)
        s.t_h, s.t_md, s.step = rep.t_h0, rep.t_md0, int(rep.step0)
        # eigenvalue bias (Eq. 13, Eq. 15): off unless the replica asks for it
        self.veig = np.zeros((n, 3))
        s.eig_on = int(getattr(rep, "eig_on", 0))
        s.eig_maxit = int(getattr(rep, "eig_maxit", 2000))
        s.eig_lo, s.eig_hi = float(getattr(rep, "eig_lo", 0.0)), float(getattr(rep, "eig_hi", 1.0))
        s.veig = _dp(self.veig)
        # continuous sliding: slider x = x_S0 + k (v dt) after the k-th step from here
        s.vslide = float(getattr(rep, "v_slide", 0.0))
        s.slide_x0, s.slide_step0 = float(rep.slider[0]), int(rep.step0)
        # harmonic tip bonds (Eq. 12); none: every pair is LJ
        b = getattr(rep, "bonds", None)
        self.bonds = np.zeros((0, 2), np.int32) if b is None else np.ascontiguousarray(b, dtype=np.int32).reshape(-1, 2)
        s.nbond = len(self.bonds)
        s.bonds = self.bonds.ctypes.data_as(C.POINTER(C.c_int))
        s.kbond, s.rbond = float(getattr(rep, "k_bond", 57.2)), float(getattr(rep, "r_bond", 1.12))
        # Nose-Hoover chain in place of Langevin (0: Langevin)
        s.nhc_len = int(getattr(rep, "nhc_len", 0))
        s.nhc_tau = float(getattr(rep, "nhc_tau", 0.5))
        if not 0 <= s.nhc_len <= 8:
            raise ValueError("nhc_len must be in [0, 8]")
        self.s = s
        self.rep = rep
        if draw_velocities is None:
            draw_velocities = rep.vel is None
        lib().or_init(C.byref(s), C.byref(self.P), int(bool(draw_velocities)))

    # ---- thin wrappers ----
    @property
    def n(self):
        return self.s.n

    def set_positions(self, x):
        self.x[...] = x

    def refresh(self):
        """Rebuild the list and recompute forces and bias at the current x."""
        L = lib()
        L.or_nlist_cells(C.byref(self.s), self.params.rc + self.params.skin)
        L.or_forces(C.byref(self.s), C.byref(self.P))
        L.or_bias_eval(C.byref(self.s), C.byref(self.P))

    def nlist_brute(self, rl=None):
        rl = self.params.rc + self.params.skin if rl is None else rl
        return lib().or_nlist_brute(C.byref(self.s), rl)

    def nlist_cells(self, rl=None):
        rl = self.params.rc + self.params.skin if rl is None else rl
        return lib().or_nlist_cells(C.byref(self.s), rl)

    def rows(self):
        return [self.nbr[i, : self.nnb[i]].copy() for i in range(self.n)]

    def forces(self):
        return lib().or_forces(C.byref(self.s), C.byref(self.P))

    def forces_brute(self):
        f = np.zeros((self.n, 3))
        e = np.zeros(self.n)
        v = lib().or_forces_brute(C.byref(self.s), C.byref(self.P), _dp(f), _dp(e))
        return f, e, v

    def potential(self, x=None):
        x = self.x if x is None else np.ascontiguousarray(x, dtype=np.float64)
        return lib().or_potential(C.byref(self.s), C.byref(self.P), _dp(x))

    def gradient(self, x=None):
        x = self.x if x is None else np.ascontiguousarray(x, dtype=np.float64)
        g = np.zeros((self.n, 3))
        lib().or_gradient(C.byref(self.s), C.byref(self.P), _dp(x), _dp(g))
        return g

    def hessvec(self, u, x=None):
        x = self.x if x is None else np.ascontiguousarray(x, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros((self.n, 3))
        lib().or_hessvec(C.byref(self.s), C.byref(self.P), _dp(x), _dp(u), _dp(out))
        return out

    def bias_potential(self, x=None):
        x = self.x if x is None else np.ascontiguousarray(x, dtype=np.float64)
        return lib().or_bias_potential(C.byref(self.s), C.byref(self.P), _dp(x))

    def bias_eval(self):
        lib().or_bias_eval(C.byref(self.s), C.byref(self.P))

    def dv1(self, sigma):
        out = np.zeros(2)
        lib().or_dv1(C.byref(self.s), float(sigma), _dp(out))
        return out

    def run(self, nsteps):
        lib().or_run(C.byref(self.s), C.byref(self.P), int(nsteps))

    def quench(self, method=0, ftol=1e-6, max_iter=20000, step_size=None, ftol_stay=0.0, keep=0.0):
        """Quench a copy of the positions; with ftol_stay > 0 the quench also
        stops once max|F| < ftol_stay with every atom within keep of r_O."""
        if step_size is None:
            step_size = (0.002 if method == 0 else 0.01)
        xq = np.zeros((self.n, 3))
        fmax = np.zeros(1)
        it = lib().or_quench_gated(C.byref(self.s), C.byref(self.P), int(method), float(ftol), float(ftol_stay),
                                   float(keep), int(max_iter), float(step_size), _dp(xq), _dp(fmax))
        return xq, int(it), float(fmax[0])

    # ---- eigenvalue bias (Eq. 13, Eq. 15) ----
    def project(self, u):
        """P u: fixed atoms (and z in 2-D) zeroed, rigid atoms set to the layer mean."""
        u = np.ascontiguousarray(u, dtype=np.float64).copy()
        lib().or_project(C.byref(self.s), _dp(u))
        return u

    def lowest_eig(self, x=None, v0=None, maxit=None, tol=1e-12):
        """(epsilon, v): lowest eigenvalue of P H P on the range of P at x (Lanczos)."""
        x = self.x if x is None else np.ascontiguousarray(x, dtype=np.float64)
        v = np.zeros((self.n, 3)) if v0 is None else np.ascontiguousarray(v0, dtype=np.float64).copy()
        e = lib().or_lowest_eig(C.byref(self.s), C.byref(self.P), _dp(x), _dp(v), int(maxit or 3 * self.n), tol)
        return e, v

    def eig_grad(self, v, x=None):
        """grad of v^T H(x) v over all 3N coordinates, v fixed."""
        x = self.x if x is None else np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        g = np.zeros((self.n, 3))
        lib().or_eig_grad(C.byref(self.s), C.byref(self.P), _dp(x), _dp(v), _dp(g))
        return g

    def dv2(self, e):
        out = np.zeros(2)
        lib().or_dv2(C.byref(self.s), float(e), _dp(out))
        return out

    def dv13(self, dv1, dv2):
        out = np.zeros(3)
        lib().or_dv13(C.byref(self.s), float(dv1), float(dv2), _dp(out))
        return out

    def nhc_energy(self):
        """The chain's part of the conserved extended energy."""
        return lib().or_nhc_energy(C.byref(self.s))

    def transition(self, xq, theta=0.5):
        md = np.zeros(1)
        f = lib().or_transition(C.byref(self.s), _dp(np.ascontiguousarray(xq)), float(theta), _dp(md))
        return bool(f), float(md[0])

    def obs(self):
        s = self.s
        return dict(step=s.step, t_md=s.t_md, t_h=s.t_h, V=s.V, K=s.K, dV=s.dV, sigma=s.sigma,
                    d=s.d, FR=s.FR, xT=list(s.xT), n_rebuild=s.n_rebuild, G=s.G,
                    fbody=list(s.fbody), vbody=list(s.vbody))


def run_batch(reps, nsteps):
    """Advance a list of OracleReplica in parallel (OpenMP over replicas)."""
    if not reps:
        return
    arr = (OrRep * len(reps))()
    for i, r in enumerate(reps):
        arr[i] = r.s
    lib().or_run_batch(arr, len(reps), C.byref(reps[0].P), int(nsteps))
    for i, r in enumerate(reps):
        r.s = arr[i]


def num_threads():
    return lib().or_num_threads()


def quench_batch(reps, method=1, ftol=1e-6, max_iter=20000, step_size=None, ftol_stay=0.0, keep=0.0):
    """Quench a list of OracleReplica in parallel (OpenMP over replicas);
    returns the quenched positions, iteration counts and final max forces.
    ftol_stay, keep: the early stop of OracleReplica.quench."""
    if step_size is None:
        step_size = (0.002 if method == 0 else 0.01)
    n = len(reps)
    if n == 0:
        return [], np.zeros(0, np.int32), np.zeros(0)
    arr = (OrRep * n)()
    for i, r in enumerate(reps):
        arr[i] = r.s
    xq = [np.zeros((r.n, 3)) for r in reps]
    ptrs = (C.POINTER(C.c_double) * n)(*[_dp(x) for x in xq])
    fmax = np.zeros(n)
    iters = np.zeros(n, np.int32)
    lib().or_quench_batch_gated(arr, n, C.byref(reps[0].P), int(method), float(ftol), float(ftol_stay), float(keep),
                                int(max_iter), float(step_size), ptrs, _dp(fmax),
                                iters.ctypes.data_as(C.POINTER(C.c_int)))
    return xq, iters, fmax
