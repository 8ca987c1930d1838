"""Shared pytest set-up: repo root on sys.path, markers, small seeded models."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU statistical test")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


def small2d(cols=12, rows=6, n_tip=13, kT=0.1, **kw):
    from paper_0909_5215_gb300 import model as M
    return M.afm2d(n_cols=cols, n_rows=rows, n_tip=n_tip, kT=kT, eps=M.PAPER_EPS_2D, **kw)


def small3d(nx=4, nz=3, radius=2.5, kT=0.1, **kw):
    from paper_0909_5215_gb300 import model as M
    return M.afm3d(nx=nx, ny=nx, nz=nz, tip_radius=radius, kT=kT, eps=M.PAPER_EPS_3D, **kw)


def thermalise(rep, amp=0.05, seed=1):
    """Displace mobile atoms (and the rigid layer as one body) by small seeded noise."""
    rng = np.random.default_rng(seed)
    r = rep.copy()
    mob = r.role == 1
    d = rng.normal(0.0, amp, size=r.pos.shape)
    if r.dim == 2:
        d[:, 2] = 0.0
    r.pos[mob] += d[mob]
    body = rng.normal(0.0, amp, size=3)
    if r.dim == 2:
        body[2] = 0.0
    r.pos[r.role == 2] += body
    return r
