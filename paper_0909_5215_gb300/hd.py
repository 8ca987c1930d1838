"""Thin Python binding of libhdslide (include/hd.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch provides the device workspace and the CUDA stream.  If the
library is not built, `lib()` raises: there is no CPU fallback.

Module-level functions carry the C names (hd_create, hd_step, ...); `Batch`
wraps one context for convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

HD_OK, HD_ERR_ARG, HD_ERR_CUDA, HD_ERR_NOMEM, HD_ERR_NUMERIC = 0, 1, 2, 3, 4
HD_ERR_TIMEOUT, HD_ERR_STATE, HD_ERR_UNIMPLEMENTED, HD_ERR_OVERFLOW = 5, 6, 7, 8
HD_FP64, HD_FP32_SPLIT = 0, 1
HD_DRIVER_AUTO, HD_DRIVER_KERNELS, HD_DRIVER_PERSISTENT = 0, 1, 2
(F_POS, F_VEL, F_FORCE, F_HDR, F_REF, F_NBR, F_NBR_COUNT, F_OBS, F_CELL, F_QPOS,
 F_ENERGY) = range(11)
OBS_FIELDS = ["step", "t_md", "t_h", "V", "K", "dV", "sigma", "d", "F_R", "x_T", "y_T", "z_T",
              "n_rebuild", "boost", "q_iter", "q_fmax", "G", "fbody_x", "fbody_y", "fbody_z",
              "vbody_x", "vbody_y", "vbody_z", "q_disp", "n_dv_zero", "n_dv_band", "n_dv_max", "q_conv",
              "x_S", "nhc_energy", "eig", "eig_iters"]
OBS_LEN = 32
STATUS_NAMES = {0: "HD_OK", 1: "HD_ERR_ARG", 2: "HD_ERR_CUDA", 3: "HD_ERR_NOMEM", 4: "HD_ERR_NUMERIC",
                5: "HD_ERR_TIMEOUT", 6: "HD_ERR_STATE", 7: "HD_ERR_UNIMPLEMENTED", 8: "HD_ERR_OVERFLOW"}


class HdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class hd_replica_desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n_atoms", C.c_int), ("rep_id", C.c_int), ("m_exp", C.c_int),
        ("pos", C.POINTER(C.c_double)), ("vel", C.POINTER(C.c_double)), ("pos_ref", C.POINTER(C.c_double)),
        ("role", C.POINTER(C.c_uint8)), ("type", C.POINTER(C.c_uint8)),
        ("box", C.c_double * 3), ("periodic", C.c_uint8 * 3), ("pad_", C.c_uint8 * 5),
        ("kT", C.c_double), ("gamma", C.c_double), ("k_spring", C.c_double), ("f_normal", C.c_double),
        ("slider", C.c_double * 2),
        ("dvmax", C.c_double), ("sig_lo", C.c_double), ("sig_hi", C.c_double),
        ("eps", (C.c_double * 2) * 2), ("sig", (C.c_double * 2) * 2),
        ("t_h0", C.c_double), ("t_md0", C.c_double), ("step0", C.c_int64),
        ("v_slide", C.c_double),
        ("n_bonds", C.c_int), ("pad2_", C.c_int), ("bonds", C.POINTER(C.c_int32)),
        ("k_bond", C.c_double), ("r_bond", C.c_double),
        ("nhc_len", C.c_int), ("pad3_", C.c_int), ("nhc_tau", C.c_double),
        ("eig_on", C.c_int), ("eig_maxit", C.c_int), ("eig_lo", C.c_double), ("eig_hi", C.c_double),
    ]


class hd_params(C.Structure):
    _fields_ = [("prec", C.c_int), ("bias_on", C.c_int), ("driver", C.c_int), ("block", C.c_int),
                ("dt", C.c_double), ("rc", C.c_double), ("skin", C.c_double), ("seed", C.c_uint64),
                ("maxnb", C.c_int), ("cell_cap", C.c_int), ("pair_kernel", C.c_int), ("pad_", C.c_int)]


SYMBOLS = ["hd_workspace_bytes", "hd_create", "hd_set_slider", "hd_set_bias", "hd_step", "hd_quench",
           "hd_read", "hd_info", "hd_timing", "hd_nlist_static", "hd_sync", "hd_destroy", "hd_last_error"]
INFO_FIELDS = ["n_rep", "natom", "maxnb", "cell_cap", "ntile", "driver", "persistent_ctas", "launches",
               "h2d_bytes", "d2h_bytes", "workspace_bytes", "reserved"]
TIMING_FIELDS = ["pair_ms", "pair_launches", "update_ms", "update_launches", "rebuild_prep_ms", "rebuild_passes",
                 "scalar_ms", "scalar_launches", "nlist_ms", "nlist_launches", "eig_ms", "eig_passes",
                 "reserved12", "reserved13", "reserved14", "reserved15"]
_lib = None


def lib(build_if_missing: bool = False):
    """Load libhdslide.so; raise if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.OUT):
        if not build_if_missing:
            raise RuntimeError("libhdslide.so is not built; run paper_0909_5215_gb300._build.build()")
        _build.build()
    L = C.CDLL(_build.OUT)
    vp, dp, sz = C.c_void_p, C.POINTER(C.c_double), C.c_size_t
    L.hd_workspace_bytes.argtypes = [C.POINTER(hd_replica_desc), C.c_int, C.POINTER(hd_params)]
    L.hd_workspace_bytes.restype = sz
    L.hd_create.argtypes = [C.POINTER(hd_replica_desc), C.c_int, C.POINTER(hd_params), vp, sz, vp, C.POINTER(vp)]
    L.hd_set_slider.argtypes = [vp, dp, C.c_int]
    L.hd_set_bias.argtypes = [vp, dp]
    L.hd_step.argtypes = [vp, C.c_int]
    L.hd_quench.argtypes = [vp, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                            C.POINTER(C.c_int32)]
    L.hd_read.argtypes = [vp, C.c_int, C.c_int, vp, sz]
    L.hd_info.argtypes = [vp, C.POINTER(C.c_int64)]
    L.hd_timing.argtypes = [vp, C.c_int, C.POINTER(C.c_double)]
    L.hd_nlist_static.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_uint8), C.c_double, C.c_int,
                                  vp, vp, vp]
    L.hd_sync.argtypes = [vp]
    L.hd_destroy.argtypes = [vp]
    L.hd_destroy.restype = None
    L.hd_last_error.argtypes = [vp]
    L.hd_last_error.restype = C.c_char_p
    for name in SYMBOLS:
        if name not in ("hd_workspace_bytes", "hd_destroy", "hd_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


# ---------------------------------------------------------------- same-name wrappers
def hd_workspace_bytes(descs, n_rep, params):
    return lib().hd_workspace_bytes(descs, n_rep, C.byref(params))


def hd_create(descs, n_rep, params, d_ws, ws_bytes, stream, ctx_out):
    return lib().hd_create(descs, n_rep, C.byref(params), C.c_void_p(d_ws), ws_bytes, C.c_void_p(stream),
                           C.byref(ctx_out))


def hd_set_slider(ctx, slider, requench_ref):
    a = np.ascontiguousarray(slider, dtype=np.float64)
    return lib().hd_set_slider(ctx, a.ctypes.data_as(C.POINTER(C.c_double)), int(requench_ref))


def hd_set_bias(ctx, bias):
    a = np.ascontiguousarray(bias, dtype=np.float64)
    return lib().hd_set_bias(ctx, a.ctypes.data_as(C.POINTER(C.c_double)))


def hd_step(ctx, n_steps):
    return lib().hd_step(ctx, int(n_steps))


def hd_quench(ctx, method, ftol, max_iter, step_size, theta, ftol_stay, adopt, flags):
    fp = None if flags is None else flags.ctypes.data_as(C.POINTER(C.c_int32))
    return lib().hd_quench(ctx, int(method), float(ftol), int(max_iter), float(step_size), float(theta),
                           float(ftol_stay), int(adopt), fp)


def hd_read(ctx, field, replica, dst):
    return lib().hd_read(ctx, int(field), int(replica), C.c_void_p(dst.ctypes.data), dst.nbytes)


def hd_info(ctx):
    out = (C.c_int64 * 12)()
    st = lib().hd_info(ctx, out)
    return st, list(out)


def hd_timing(ctx, enable):
    out = (C.c_double * 16)()
    st = lib().hd_timing(ctx, int(enable), out)
    return st, list(out)


def hd_nlist_static(d_pos, n_atoms, box, periodic, rl, maxnb, d_nbr, d_nnb, stream):
    """List build on caller buffers with no device allocation (device pointers as ints)."""
    b = (C.c_double * 3)(*[float(v) for v in box])
    p = (C.c_uint8 * 3)(*[int(v) for v in periodic])
    return lib().hd_nlist_static(C.c_void_p(d_pos), int(n_atoms), b, p, float(rl), int(maxnb), C.c_void_p(d_nbr),
                                 C.c_void_p(d_nnb), C.c_void_p(stream))


def hd_sync(ctx):
    return lib().hd_sync(ctx)


def hd_destroy(ctx):
    lib().hd_destroy(ctx)


def hd_last_error(ctx):
    return lib().hd_last_error(ctx).decode()


# ---------------------------------------------------------------- convenience
def make_params(params, driver=HD_DRIVER_AUTO, block=0, maxnb=0, cell_cap=0, prec=None, pair_kernel=0):
    return hd_params(int(params.prec if prec is None else prec), int(params.bias_on), int(driver), int(block),
                     float(params.dt), float(params.rc), float(params.skin), int(params.seed), int(maxnb),
                     int(cell_cap), int(pair_kernel), 0)


def make_descs(reps):
    """Build the C descriptors; returns (array, keep-alive list)."""
    keep = []
    arr = (hd_replica_desc * len(reps))()

    def dptr(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_double))

    def bptr(a):
        a = np.ascontiguousarray(a, dtype=np.uint8)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_uint8))

    for k, r in enumerate(reps):
        d = arr[k]
        d.dim, d.n_atoms, d.rep_id, d.m_exp = int(r.dim), int(r.n), int(r.rep_id), int(r.m_exp)
        d.pos = dptr(r.pos)
        d.vel = dptr(r.vel) if r.vel is not None else None
        d.pos_ref = dptr(r.pos_ref) if r.pos_ref is not None else None
        d.role, d.type = bptr(r.role), bptr(r.type)
        for a in range(3):
            d.box[a] = float(r.box[a])
            d.periodic[a] = int(r.periodic[a])
        d.kT, d.gamma, d.k_spring, d.f_normal = r.kT, r.gamma, r.k_spring, r.f_normal
        d.slider[0], d.slider[1] = float(r.slider[0]), float(r.slider[1])
        d.dvmax, d.sig_lo, d.sig_hi = r.dvmax, r.sig_lo, r.sig_hi
        for a in range(2):
            for b in range(2):
                d.eps[a][b] = float(r.eps[a][b])
                d.sig[a][b] = float(r.sig[a][b])
        d.t_h0, d.t_md0, d.step0 = float(r.t_h0), float(r.t_md0), int(r.step0)
        d.v_slide = float(getattr(r, "v_slide", 0.0))
        bonds = getattr(r, "bonds", None)
        if bonds is not None and len(bonds):
            bnd = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
            keep.append(bnd)
            d.n_bonds = len(bnd)
            d.bonds = bnd.ctypes.data_as(C.POINTER(C.c_int32))
            d.k_bond, d.r_bond = float(r.k_bond), float(r.r_bond)
        d.nhc_len = int(getattr(r, "nhc_len", 0))
        d.nhc_tau = float(getattr(r, "nhc_tau", 0.5))
        d.eig_on = int(getattr(r, "eig_on", 0))
        d.eig_maxit = int(getattr(r, "eig_maxit", 0))
        d.eig_lo, d.eig_hi = float(getattr(r, "eig_lo", 0.0)), float(getattr(r, "eig_hi", 1.0))
    return arr, keep


def workspace_bytes(reps, params, **kw) -> int:
    descs, _keep = make_descs(reps)
    return int(hd_workspace_bytes(descs, len(reps), make_params(params, **kw)))


class Batch:
    """One library context over a batch of replicas on one GPU."""

    def __init__(self, reps, params, driver=HD_DRIVER_AUTO, block=0, maxnb=0, cell_cap=0, prec=None,
                 device="cuda:0", stream=None, pair_kernel=0):
        import torch
        self.reps = reps
        self.n_rep = len(reps)
        self.ns = [r.n for r in reps]
        self.torch = torch
        self.device = torch.device(device)
        self.params = make_params(params, driver, block, maxnb, cell_cap, prec, pair_kernel)
        self.prec = self.params.prec
        descs, keep = make_descs(reps)
        nb = hd_workspace_bytes(descs, len(reps), self.params)
        if nb == 0:
            raise HdError(HD_ERR_ARG, "invalid batch (hd_workspace_bytes returned 0)")
        self.ws_bytes = int(nb)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = (self.ws.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.ctx = C.c_void_p()
        st = hd_create(descs, len(reps), self.params, base, self.ws_bytes, self.stream.cuda_stream, self.ctx)
        del keep
        if st != HD_OK:
            msg = hd_last_error(self.ctx)
            hd_destroy(self.ctx)
            self.ctx = None
            raise HdError(st, msg)
        _, info = hd_info(self.ctx)
        self.maxnb = info[2]

    # ---- calls
    def _ck(self, st):
        if st != HD_OK:
            raise HdError(st, hd_last_error(self.ctx))

    def step(self, n):
        self._ck(hd_step(self.ctx, n))

    def sync(self):
        self._ck(hd_sync(self.ctx))

    def set_slider(self, slider, requench_ref=0):
        self._ck(hd_set_slider(self.ctx, np.asarray(slider, dtype=np.float64).reshape(-1), requench_ref))

    def set_bias(self, bias):
        self._ck(hd_set_bias(self.ctx, np.asarray(bias, dtype=np.float64).reshape(-1)))

    def quench(self, method=1, ftol=1e-6, max_iter=20000, step_size=None, theta=0.5, adopt=0, ftol_stay=0.0):
        """hd_quench; returns the transition flags.  ftol_stay > ftol stops a
        replica early once max|F| < ftol_stay with every atom within theta/2
        of r_O."""
        if step_size is None:
            step_size = 0.002 if method == 0 else 0.005
        flags = np.zeros(self.n_rep, dtype=np.int32)
        self._ck(hd_quench(self.ctx, method, ftol, max_iter, step_size, theta, ftol_stay, adopt, flags))
        self.last_flags = flags
        return flags

    def qstats(self):
        """Iterations (mean, max), largest final force of the replicas that
        reached ftol, that stopped inside their basin and that did neither,
        their fractions, and the number of flagged replicas of the last
        quench."""
        ob = self.obs()
        cv = ob[:, 27]
        return {"iters": float(ob[:, 14].mean()), "iters_max": int(ob[:, 14].max()),
                "fmax": float(ob[cv == 1, 15].max()) if (cv == 1).any() else 0.0,
                "fmax_stay": float(ob[cv == 2, 15].max()) if (cv == 2).any() else 0.0,
                "fmax_unconverged": float(ob[cv == 0, 15].max()) if (cv == 0).any() else 0.0,
                "converged": float((cv == 1).mean()), "stayed": float((cv == 2).mean()),
                "flagged": int(getattr(self, "last_flags", np.zeros(1)).sum())}

    def _read(self, field, r, shape, dtype):
        out = np.empty(shape, dtype=dtype)
        self._ck(hd_read(self.ctx, field, r, out))
        return out

    def positions(self, r):
        return self._read(F_POS, r, (self.ns[r], 3), np.float64)

    def velocities(self, r):
        return self._read(F_VEL, r, (self.ns[r], 3), np.float64)

    def forces(self, r):
        return self._read(F_FORCE, r, (self.ns[r], 3), np.float64)

    def energies(self, r):
        return self._read(F_ENERGY, r, (self.ns[r],), np.float64)

    def hdr(self, r):
        return self._read(F_HDR, r, (self.ns[r], 3), np.float64)

    def ref(self, r):
        return self._read(F_REF, r, (self.ns[r], 3), np.float64)

    def qpos(self, r):
        return self._read(F_QPOS, r, (self.ns[r], 3), np.float64)

    def nbr_count(self, r):
        return self._read(F_NBR_COUNT, r, (self.ns[r],), np.int32)

    def nbr(self, r):
        return self._read(F_NBR, r, (self.ns[r], self.maxnb), np.int32)

    def rows(self, r):
        cnt, nb = self.nbr_count(r), self.nbr(r)
        return [nb[i, : cnt[i]].copy() for i in range(self.ns[r])]

    def cells(self, r):
        return self._read(F_CELL, r, (self.ns[r],), np.int32)

    def obs(self, r=None):
        if r is None:
            a = self._read(F_OBS, -1, (self.n_rep, OBS_LEN), np.float64)
            return a
        a = self._read(F_OBS, r, (OBS_LEN,), np.float64)
        return dict(zip(OBS_FIELDS, a.tolist()))

    def info(self):
        st, inf = hd_info(self.ctx)
        self._ck(st)
        return dict(zip(INFO_FIELDS, inf))

    def timing(self, enable=-1):
        """CUDA-event totals of the pair kernel and the other phases (ms, counts)."""
        st, out = hd_timing(self.ctx, enable)
        self._ck(st)
        return dict(zip(TIMING_FIELDS, out))

    def close(self):
        if self.ctx:
            hd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
