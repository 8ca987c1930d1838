"""Seeded input generator for the AFM sliding models (geometry only).

This module builds the inputs that both the CUDA path and the CPU oracle
consume: atom positions, roles, types, boxes and per-replica settings.  It
holds none of the method's arithmetic (no potential, no bias, no integrator,
no random draws of the method); velocities are drawn by the method itself
from its counter-based generator.

Models (Kim & Falk, Sec. 3.1.1 and Sec. 3.2.1):

* 2-D: a triangular-lattice substrate (nearest-neighbour spacing 2^(1/6)),
  periodic along x, bottom rows fixed, with a half-disc tip carved from the
  same lattice continued above the substrate, so the tip sits in registry
  with it (Sec. 3.1.1).  The flat top row of the tip is the rigid layer that
  the slider spring pulls and the normal load pushes (Sec. 3.1.1).
* 3-D: an fcc substrate of cubic 4-atom cells joined along [001], periodic
  in x and y, bottom atomic layers fixed, with a hemispherical tip carved
  from the same fcc lattice (Sec. 3.2.1); its flat top layer is rigid.

Roles: 0 fixed, 1 mobile, 2 rigid (top layer of the tip).
Types: 0 substrate, 1 tip (the LJ parameter pair of Eq. 9 is chosen by type).

Readings where the paper is silent:
* The 2-D tip is the set of lattice sites within radius R of a centre placed
  R above the apex site (the apex is the tip site right above the substrate
  near the box centre), with R grown in steps of 0.01 until at least n_tip
  sites are inside; surplus sites are dropped farthest-from-centre first
  (the apex is always kept; ties drop the larger site index).
* The 3-D tip is the set of fcc sites within radius R of a centre R above
  the apex site, cut at the highest full lattice layer below the centre.
* Atoms are emitted in a spatially blocked (Morton) order of 1.4-sigma
  cells so that atoms close in space are close in memory.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ROLE_FIXED, ROLE_MOBILE, ROLE_RIGID = 0, 1, 2
TYPE_SUB, TYPE_TIP = 0, 1

PAPER_EPS_2D = ((1.0, 0.5), (0.5, 1.0))     # Sec. 3.1.1: eps_ss = eps_tt = 1, eps_ts = 0.5
PAPER_EPS_3D = ((1.0, 0.2), (0.2, 1.0))     # Sec. 3.2.1: eps_ss = 1, eps_st = 0.2 (tip-tip LJ, eps 1)

A2D = 2.0 ** (1.0 / 6.0)          # 2-D nearest-neighbour spacing (LJ minimum)
AFCC = 2.0 ** (2.0 / 3.0)         # fcc cubic lattice constant, nn = 2^(1/6)


@dataclass
class Replica:
    """One AFM model at one slider position (all arrays host, FP64/uint8)."""
    dim: int
    pos: np.ndarray                 # (n, 3) float64; z == 0 in 2-D
    role: np.ndarray                # (n,) uint8
    type: np.ndarray                # (n,) uint8
    box: np.ndarray                 # (3,) float64 periodic lengths (0 if open)
    periodic: np.ndarray            # (3,) uint8
    kT: float = 0.05
    gamma: float = 1.0
    k_spring: float = 1.0
    f_normal: float = 1.0
    slider: np.ndarray = field(default_factory=lambda: np.zeros(2))
    dvmax: float = 0.0
    sig_lo: float = 0.0
    sig_hi: float = 0.0
    m_exp: int = 2
    rep_id: int = 0
    eps: tuple = ((1.0, 0.5), (0.5, 1.0))   # LJ energy per type pair, Eq. 9
    sig: tuple = ((1.0, 1.0), (1.0, 1.0))   # LJ length per type pair, Eq. 9
    vel: np.ndarray | None = None   # (n, 3) or None -> Maxwell-Boltzmann
    pos_ref: np.ndarray | None = None  # (n, 3) reference minimum or None
    t_h0: float = 0.0
    t_md0: float = 0.0
    step0: int = 0
    # eigenvalue bias (Eq. 13, Eq. 15): band [eig_lo, eig_hi] of the lowest
    # Hessian eigenvalue; evaluated by the CPU oracle only so far
    eig_on: int = 0
    eig_lo: float = 0.0
    eig_hi: float = 1.0
    eig_maxit: int = 2000          # Lanczos steps per evaluation, at most (capped at the allowed dimension)
    # continuous sliding (slider moving at v_slide along x every step);
    # evaluated by the CPU oracle only so far
    v_slide: float = 0.0
    # harmonic tip bonds (Eq. 12): (m, 2) atom pairs bonded by
    # k_bond (r - r_bond)^2 / 2; with bonds the tip-tip LJ term is dropped.
    # Evaluated by the CPU oracle only so far.
    bonds: np.ndarray | None = None
    k_bond: float = 57.2
    r_bond: float = 1.12
    # Nose-Hoover chain (length nhc_len, period nhc_tau) in place of Langevin;
    # 0: Langevin.  Evaluated by the CPU oracle only so far.
    nhc_len: int = 0
    nhc_tau: float = 0.5

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def tip_com(self) -> np.ndarray:
        """Centre of the rigid layer (the tip position x_T of Sec. 3.1.2)."""
        return self.pos[self.role == ROLE_RIGID].mean(axis=0)

    def copy(self) -> "Replica":
        r = Replica(**{k: (v.copy() if isinstance(v, np.ndarray) else v)
                       for k, v in self.__dict__.items()})
        return r


@dataclass
class Params:
    """Global parameters shared by all replicas of one batch."""
    dt: float = 0.005
    rc: float = 2.5
    skin: float = 0.3
    bias_on: int = 0
    seed: int = 20250909
    prec: int = 0                            # 0 FP64, 1 FP32 split


def _morton_order(pos: np.ndarray, cell: float = 1.4) -> np.ndarray:
    q = np.floor((pos - pos.min(axis=0)) / cell).astype(np.int64)
    key = np.zeros(len(pos), dtype=np.int64)
    for bit in range(20):
        for d in range(3):
            key |= ((q[:, d] >> bit) & 1) << (3 * bit + d)
    return np.argsort(key, kind="stable")


def _finish(dim, pos, role, typ, box, periodic, **kw) -> Replica:
    order = _morton_order(pos)
    rep = Replica(dim=dim, pos=np.ascontiguousarray(pos[order], dtype=np.float64),
                  role=np.ascontiguousarray(role[order], dtype=np.uint8),
                  type=np.ascontiguousarray(typ[order], dtype=np.uint8),
                  box=np.asarray(box, dtype=np.float64),
                  periodic=np.asarray(periodic, dtype=np.uint8), **kw)
    com = rep.tip_com()
    if "slider" not in kw:
        rep.slider = np.array([com[0], com[1]], dtype=np.float64)
    return rep


def afm2d(n_cols: int = 48, n_rows: int = 8, n_fixed_rows: int = 2,
          n_tip: int = 37, **kw) -> Replica:
    """2-D triangular-lattice substrate plus half-disc tip (Sec. 3.1.1)."""
    dy = A2D * math.sqrt(3.0) / 2.0
    lx = n_cols * A2D
    sub = []
    for j in range(n_rows):
        for i in range(n_cols):
            sub.append(((i + 0.5 * (j % 2)) * A2D, j * dy))
    sub = np.array(sub)
    sub_role = np.where(np.arange(len(sub)) // n_cols < n_fixed_rows,
                        ROLE_FIXED, ROLE_MOBILE)
    # tip sites: lattice continued above the substrate
    ja = n_rows
    ia = int(round(lx / 2.0 / A2D - 0.5 * (ja % 2)))
    apex = np.array([(ia + 0.5 * (ja % 2)) * A2D, ja * dy])
    cand = []
    for j in range(ja, ja + 64):
        for i in range(n_cols):
            cand.append(((i + 0.5 * (j % 2)) * A2D, j * dy))
    cand = np.array(cand)
    apex_idx = int(np.argmin(((cand - apex) ** 2).sum(1)))
    radius = A2D
    while True:
        centre = apex + np.array([0.0, radius])
        d2 = ((cand - centre) ** 2).sum(1)
        inside = (d2 <= radius * radius * (1 + 1e-12)) & (cand[:, 1] <= centre[1] + 1e-9)
        if inside.sum() >= n_tip:
            break
        radius += 0.01
    idx = np.nonzero(inside)[0]
    surplus = len(idx) - n_tip
    if surplus > 0:
        others = [k for k in idx if k != apex_idx]
        others.sort(key=lambda k: (-d2[k], -k))
        drop = set(others[:surplus])
        idx = np.array([k for k in idx if k not in drop])
    tip = cand[idx]
    ytop = tip[:, 1].max()
    tip_role = np.where(np.abs(tip[:, 1] - ytop) < 1e-9, ROLE_RIGID, ROLE_MOBILE)
    pos = np.zeros((len(sub) + len(tip), 3))
    pos[: len(sub), :2] = sub
    pos[len(sub):, :2] = tip
    role = np.concatenate([sub_role, tip_role]).astype(np.uint8)
    typ = np.concatenate([np.full(len(sub), TYPE_SUB), np.full(len(tip), TYPE_TIP)]).astype(np.uint8)
    return _finish(2, pos, role, typ, (lx, 0.0, 0.0), (1, 0, 0), **kw)


def afm3d(nx: int = 24, ny: int = 24, nz: int = 6, n_fixed_layers: int = 2,
          tip_radius: float = 6.0, **kw) -> Replica:
    """3-D fcc [001] substrate plus hemispherical tip (Sec. 3.2.1)."""
    a = AFCC
    basis = np.array([(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)])
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    sub = ((g[:, None, :] + basis[None]) * a).reshape(-1, 3)
    layer = np.rint(sub[:, 2] / (a / 2)).astype(int)
    sub_role = np.where(layer < n_fixed_layers, ROLE_FIXED, ROLE_MOBILE)
    ztop_sub = sub[:, 2].max()
    za = ztop_sub + a / 2
    cx, cy = nx * a / 2, ny * a / 2
    nr = int(tip_radius / a) + 3
    ic, jc = int(round(cx / a)), int(round(cy / a))
    kz0 = int(round(za / a)) - 1
    gt = np.stack(np.meshgrid(np.arange(ic - nr, ic + nr + 1), np.arange(jc - nr, jc + nr + 1),
                              np.arange(kz0, kz0 + 2 * nr + 2), indexing="ij"), -1).reshape(-1, 3)
    cand = ((gt[:, None, :] + basis[None]) * a).reshape(-1, 3)
    cand = cand[cand[:, 2] >= za - 1e-9]
    lay = cand[np.abs(cand[:, 2] - za) < 1e-9]
    apex = lay[np.argmin((lay[:, 0] - cx) ** 2 + (lay[:, 1] - cy) ** 2)]
    centre = apex + np.array([0.0, 0.0, tip_radius])
    d2 = ((cand - centre) ** 2).sum(1)
    tip = cand[(d2 <= tip_radius ** 2 * (1 + 1e-12)) & (cand[:, 2] <= centre[2] + 1e-9)]
    ztop = tip[:, 2].max()
    tip_role = np.where(np.abs(tip[:, 2] - ztop) < 1e-9, ROLE_RIGID, ROLE_MOBILE)
    pos = np.concatenate([sub, tip])
    role = np.concatenate([sub_role, tip_role]).astype(np.uint8)
    typ = np.concatenate([np.full(len(sub), TYPE_SUB), np.full(len(tip), TYPE_TIP)]).astype(np.uint8)
    return _finish(3, pos, role, typ, (nx * a, ny * a, 0.0), (1, 1, 0), **kw)


def paper2d(**kw) -> Replica:
    """The paper's own 2-D model (Sec. 3.1.1): 80 substrate and 33 tip atoms,
    k = 5, F_N = 5, eps_ts = 0.5.  Reading (the figure is not available): the
    substrate is 20 columns x 4 rows of the triangular lattice with the bottom
    row fixed; the tip is an inverted trapezoid of rows holding 3, 4, ..., 8
    atoms on the lattice sites continued above the substrate (so its contact
    row is in registry), the top row of 8 rigid."""
    n_cols, n_rows = 20, 4
    dy = A2D * math.sqrt(3.0) / 2.0
    lx = n_cols * A2D
    sub = np.array([((i + 0.5 * (j % 2)) * A2D, j * dy) for j in range(n_rows) for i in range(n_cols)])
    sub_role = np.where(np.arange(len(sub)) < n_cols, ROLE_FIXED, ROLE_MOBILE)
    ja = n_rows
    ia = int(round(lx / 2.0 / A2D - 0.5 * (ja % 2)))
    xc = (ia + 0.5 * (ja % 2)) * A2D
    tip, tip_role = [], []
    for k, m in enumerate(range(3, 9)):
        for q in range(m):
            tip.append((xc + (q - 0.5 * (m - 1)) * A2D, (ja + k) * dy))
            tip_role.append(ROLE_RIGID if m == 8 else ROLE_MOBILE)
    tip = np.array(tip)
    pos = np.zeros((len(sub) + len(tip), 3))
    pos[: len(sub), :2] = sub
    pos[len(sub):, :2] = tip
    role = np.concatenate([sub_role, tip_role]).astype(np.uint8)
    typ = np.concatenate([np.full(len(sub), TYPE_SUB), np.full(len(tip), TYPE_TIP)]).astype(np.uint8)
    kw.setdefault("k_spring", 5.0)
    kw.setdefault("f_normal", 5.0)
    kw.setdefault("eps", PAPER_EPS_2D)
    return _finish(2, pos, role, typ, (lx, 0.0, 0.0), (1, 0, 0), **kw)


def tip_bonds(rep: Replica, cut: float = 1.3) -> np.ndarray:
    """Nearest-neighbour pairs of tip atoms (distance < cut) in the given
    configuration, each once (i < j)."""
    t = np.nonzero(rep.type == TYPE_TIP)[0]
    x = rep.pos[t]
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    a, b = np.nonzero(np.triu(d2 < cut * cut, 1))
    return np.stack([t[a], t[b]], 1).astype(np.int32)


def paper3d(**kw) -> Replica:
    """The paper's own 3-D model (Sec. 3.2.1): 1800 fcc substrate atoms and a
    183-atom tip joined along [001], k = 10, F_N = 5, eps_st = 0.2, tip atoms
    held together by harmonic bonds (Eq. 12, k = 57.2, r_O = 1.12) instead of
    LJ.  Reading (the figure is not available): the substrate is 15 x 15 x 2
    cubic cells (four atomic layers, the bottom one fixed); the tip is a cone
    with flat ends on the fcc sites continued above the substrate: in the
    k-th layer (k = 0 at the contact) the sites within 1.08 a + 0.42 a k of
    the axis, which gives layers of 9, 16, 21, 32, 45 and 60 atoms (the nine
    contact atoms in registry with the substrate), the top layer rigid; bonds
    join tip atoms at the nearest-neighbour distance."""
    a = AFCC
    nx = ny = 15
    basis = np.array([(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)])
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(2), indexing="ij"), -1).reshape(-1, 3)
    sub = ((g[:, None, :] + basis[None]) * a).reshape(-1, 3)
    layer = np.rint(sub[:, 2] / (a / 2)).astype(int)
    sub_role = np.where(layer < 1, ROLE_FIXED, ROLE_MOBILE)
    za = sub[:, 2].max() + a / 2
    # apex: the site of the first layer above the substrate nearest the centre
    k0 = int(round(za / (a / 2)))
    cx, cy = nx * a / 2, ny * a / 2
    best = None
    for i in range(2 * nx):
        for j in range(2 * ny):
            if (i + j + k0) % 2 == 0:
                d = (i * a / 2 - cx) ** 2 + (j * a / 2 - cy) ** 2
                if best is None or d < best[0]:
                    best = (d, i, j)
    _, i0, j0 = best
    tip, tip_role = [], []
    for k in range(6):
        rmax = 1.08 * a + 0.42 * a * k
        n = int(rmax / (a / 2)) + 1
        for i in range(i0 - n, i0 + n + 1):
            for j in range(j0 - n, j0 + n + 1):
                if (i + j + k0 + k) % 2:
                    continue
                dx, dy2 = (i - i0) * a / 2, (j - j0) * a / 2
                if dx * dx + dy2 * dy2 <= rmax * rmax * (1 + 1e-12):
                    tip.append((i * a / 2, j * a / 2, za + k * a / 2))
                    tip_role.append(ROLE_RIGID if k == 5 else ROLE_MOBILE)
    tip = np.array(tip)
    pos = np.concatenate([sub, tip])
    role = np.concatenate([sub_role, tip_role]).astype(np.uint8)
    typ = np.concatenate([np.full(len(sub), TYPE_SUB), np.full(len(tip), TYPE_TIP)]).astype(np.uint8)
    kw.setdefault("k_spring", 10.0)
    kw.setdefault("f_normal", 5.0)
    kw.setdefault("eps", PAPER_EPS_3D)
    rep = _finish(3, pos, role, typ, (nx * a, ny * a, 0.0), (1, 1, 0), **kw)
    rep.bonds = tip_bonds(rep)
    return rep


# --------------------------------------------------------------------------
# Workloads.  Each returns (list[Replica], Params).
# --------------------------------------------------------------------------

def afm2d_plain(seed: int = 20250909, prec: int = 0):
    """2-D model, one slider position, no bias; ~421 atoms, T=0.05 (the plain
    FP64 configuration; prec selects the form)."""
    r = afm2d(kT=0.05, gamma=1.0, k_spring=1.0, f_normal=1.0, rep_id=0, eps=PAPER_EPS_2D)
    return [r], Params(bias_on=0, seed=seed, prec=prec)


def afm2d_hyper(n_rep: int = 16, spacing: float = 0.05, prec: int = 1, seed: int = 20250909):
    """The 2-D model at n_rep slider positions spaced `spacing`, bias on."""
    base = afm2d(kT=0.05, gamma=1.0, k_spring=1.0, f_normal=1.0, eps=PAPER_EPS_2D)
    reps = []
    for i in range(n_rep):
        r = base.copy()
        r.rep_id = i
        r.slider = base.slider + np.array([spacing * i, 0.0])
        r.dvmax = 4.0 * r.kT
        reps.append(r)
    return reps, Params(bias_on=1, seed=seed, prec=prec)


def afm3d_hyper(n_rep: int = 64, spacing: float = 0.02, nx: int = 24, nz: int = 6,
                tip_radius: float = 6.0, kT: float = 0.1, prec: int = 1, seed: int = 20250909):
    """3-D fcc slab nx*nx*nz cells plus hemispherical tip, n_rep slider positions."""
    base = afm3d(nx=nx, ny=nx, nz=nz, tip_radius=tip_radius, kT=kT, gamma=1.0,
                 k_spring=1.0, f_normal=1.0, eps=PAPER_EPS_3D)
    reps = []
    for i in range(n_rep):
        r = base.copy()
        r.rep_id = i
        r.slider = base.slider + np.array([spacing * i, 0.0])
        r.dvmax = 4.0 * r.kT
        reps.append(r)
    return reps, Params(bias_on=1, seed=seed, prec=prec)


def afm3d_large(n_rep: int = 32, prec: int = 1, seed: int = 20250909):
    """Large 3-D model: 64x64x10 cells plus radius-12 tip, 32 slider positions."""
    return afm3d_hyper(n_rep=n_rep, spacing=0.02, nx=64, nz=10, tip_radius=12.0,
                       kT=0.1, prec=prec, seed=seed)


def uneven_batch(n_rep: int = 192, seed: int = 4, prec: int = 1,
                 n2d=(400, 4000), n3d=(5000, 40000)):
    """Uneven batch: each replica drawn from `seed` (dimension, size, T, x_S).

    Dimension ~ Bernoulli(1/2); 2-D sizes log-uniform in n2d (strip of 8 rows,
    width chosen from the size), 3-D sizes log-uniform in n3d (slab of 6 cell
    layers, square footprint chosen from the size, radius-6 tip); T uniform in
    [0.05, 0.15]; slider offset uniform in [0, 1.12].
    """
    rng = np.random.default_rng(seed)
    reps = []
    cache = {}
    for i in range(n_rep):
        dim = 2 if rng.random() < 0.5 else 3
        lo, hi = (n2d if dim == 2 else n3d)
        n = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        kT = float(rng.uniform(0.05, 0.15))
        off = float(rng.uniform(0.0, 1.12))
        if dim == 2:
            cols = max(8, int(round((n - 37) / 8)))
            key = (2, cols)
            if key not in cache:
                cache[key] = afm2d(n_cols=cols, eps=PAPER_EPS_2D)
        else:
            side = max(5, int(round(math.sqrt(max(n - 448, 1) / 24.0))))
            key = (3, side)
            if key not in cache:
                cache[key] = afm3d(nx=side, ny=side, nz=6, eps=PAPER_EPS_3D)
        r = cache[key].copy()
        r.kT, r.rep_id = kT, i
        r.slider = r.slider + np.array([off, 0.0])
        r.dvmax = 4.0 * kT
        reps.append(r)
    return reps, Params(bias_on=1, seed=seed, prec=prec)


WORKLOADS = {
    "afm2d_plain": afm2d_plain,
    "afm2d_hyper16": afm2d_hyper,
    "afm3d_hyper64": afm3d_hyper,
    "uneven192": uneven_batch,
    "afm3d_large32": afm3d_large,
}
