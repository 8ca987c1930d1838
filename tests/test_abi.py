"""The C-ABI library builds, loads and exports what include/hd.h declares.

No GPU: only host-side logic is exercised (workspace sizing, argument
checks that return before any CUDA call) plus the binding's struct layout,
checked against the C compiler's view of include/hd.h.
"""
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT, small2d, small3d

HDR = os.path.join(ROOT, "include", "hd.h")


@pytest.fixture(scope="module")
def hdlib():
    from paper_0909_5215_gb300 import _build, hd
    _build.build()
    return hd


def declared_functions():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hd_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hd_create", "hd_set_slider", "hd_step", "hd_quench", "hd_read"):
        assert must in names


def test_library_exports_every_declared_symbol(hdlib):
    out = subprocess.run(["nm", "-D", "--defined-only", hdlib._build.OUT], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (hd_[a-z_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = hdlib.lib()
    for n in declared_functions():
        assert hasattr(L, n)
    assert set(hdlib.SYMBOLS) <= set(declared_functions())


def test_struct_layout_matches_header(hdlib, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "hd.h"
#define F(T, m) printf("%s.%s %zu\n", #T, #m, offsetof(T, m))
int main(void) {
  printf("sizeof.hd_replica_desc %zu\nsizeof.hd_params %zu\n", sizeof(hd_replica_desc), sizeof(hd_params));
  F(hd_replica_desc, pos); F(hd_replica_desc, role); F(hd_replica_desc, box); F(hd_replica_desc, periodic);
  F(hd_replica_desc, kT); F(hd_replica_desc, slider); F(hd_replica_desc, dvmax); F(hd_replica_desc, eps);
  F(hd_replica_desc, sig); F(hd_replica_desc, t_h0); F(hd_replica_desc, step0);
  F(hd_params, dt); F(hd_params, seed); F(hd_params, maxnb); F(hd_params, cell_cap);
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HDR), "-o", str(exe), str(src)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    import ctypes as C
    D, P = hdlib.hd_replica_desc, hdlib.hd_params
    assert int(got["sizeof.hd_replica_desc"]) == C.sizeof(D)
    assert int(got["sizeof.hd_params"]) == C.sizeof(P)
    for key, val in got.items():
        kind, field = key.split(".")
        if kind == "sizeof":
            continue
        cls = D if kind == "hd_replica_desc" else P
        assert getattr(cls, field).offset == int(val), key


def test_workspace_sizing_host_only(hdlib):
    from paper_0909_5215_gb300 import model as M
    reps = [small2d(), small3d()]
    p = M.Params(prec=1)
    nb = hdlib.workspace_bytes(reps, p)
    n = sum(r.n for r in reps)
    assert nb > n * (3 * 32 + 112 * 4) and nb % 256 == 0
    # FP64 form holds wider velocity/force arrays
    assert hdlib.workspace_bytes(reps, M.Params(prec=0)) > nb
    # invalid batches size to 0
    bad = small2d()
    bad.role = bad.role.copy()
    bad.role[0] = 7
    assert hdlib.workspace_bytes([bad], p) == 0
    bad = small3d()
    bad.periodic = np.array([1, 1, 1], dtype=np.uint8)
    assert hdlib.workspace_bytes([bad], p) == 0
    assert hdlib.workspace_bytes([small2d()], M.Params(dt=-1.0)) == 0
    assert hdlib.workspace_bytes([small2d()], p, block=100) == 0
    assert hdlib.workspace_bytes([small2d()], p, maxnb=1000) == 0


def test_empty_and_degenerate_batches_size_to_zero(hdlib):
    """The host checks that run before any device work: no replicas, a
    replica without atoms, non-finite or out-of-plane positions, bad roles,
    types or temperatures all give 0 bytes (hd_create: HD_ERR_ARG)."""
    from paper_0909_5215_gb300 import model as M
    p = M.Params(prec=1)
    descs, keep = hdlib.make_descs([small2d()])
    assert hdlib.hd_workspace_bytes(descs, 0, hdlib.make_params(p)) == 0
    del keep

    def sized(mutate):
        r = small2d()
        r.pos, r.role, r.type = r.pos.copy(), r.role.copy(), r.type.copy()
        mutate(r)
        return hdlib.workspace_bytes([r], p)

    assert sized(lambda r: None) > 0
    def empty(r):
        r.pos, r.role, r.type = r.pos[:0], r.role[:0], r.type[:0]
    assert sized(empty) == 0
    assert sized(lambda r: r.pos.__setitem__((3, 0), np.nan)) == 0
    assert sized(lambda r: r.pos.__setitem__((3, 1), np.inf)) == 0
    assert sized(lambda r: r.pos.__setitem__((3, 2), 0.5)) == 0         # 2-D needs z == 0
    assert sized(lambda r: r.type.__setitem__(0, 2)) == 0
    assert sized(lambda r: setattr(r, "kT", 0.0)) == 0
    assert sized(lambda r: setattr(r, "m_exp", 0)) == 0


def test_create_rejects_bad_arguments_before_any_device_work(hdlib):
    import ctypes as C
    from paper_0909_5215_gb300 import model as M
    reps = [small2d()]
    descs, keep = hdlib.make_descs(reps)
    prm = hdlib.make_params(M.Params(prec=1))
    ctx = C.c_void_p()
    # NULL workspace
    st = hdlib.hd_create(descs, 1, prm, 0, 1 << 20, 0, ctx)
    assert st == hdlib.HD_ERR_ARG and "workspace" in hdlib.hd_last_error(ctx)
    hdlib.hd_destroy(ctx)
    # too small a workspace (a fake, never dereferenced, aligned address)
    ctx = C.c_void_p()
    st = hdlib.hd_create(descs, 1, prm, 1 << 20, 256, 0, ctx)
    assert st == hdlib.HD_ERR_NOMEM
    hdlib.hd_destroy(ctx)
    # misaligned workspace
    ctx = C.c_void_p()
    st = hdlib.hd_create(descs, 1, prm, (1 << 20) + 8, 1 << 30, 0, ctx)
    assert st == hdlib.HD_ERR_ARG
    hdlib.hd_destroy(ctx)
    del keep


def test_binding_fails_loudly_without_library(hdlib, monkeypatch):
    from paper_0909_5215_gb300 import _build
    monkeypatch.setattr(_build, "OUT", "/nonexistent/libhdslide.so")
    monkeypatch.setattr(hdlib, "_lib", None)
    with pytest.raises(RuntimeError):
        hdlib.lib()


def test_eigenvalue_bias_reaches_the_descriptor(hdlib):
    """The eigenvalue bias (Eq. 13, Eq. 15) is carried into the C descriptor;
    a band with eig_lo >= eig_hi is refused on the host."""
    from conftest import small2d
    from paper_0909_5215_gb300 import model as M
    r = small2d()
    r.eig_on, r.eig_lo, r.eig_hi, r.eig_maxit = 1, 0.5, 2.0, 300
    descs, _keep = hdlib.make_descs([r])
    assert descs[0].eig_on == 1 and descs[0].eig_lo == 0.5 and descs[0].eig_hi == 2.0 and descs[0].eig_maxit == 300
    assert hdlib.hd_workspace_bytes(descs, 1, hdlib.make_params(M.Params(bias_on=1))) > 0
    r.eig_lo = 3.0
    descs, _keep = hdlib.make_descs([r])
    assert hdlib.hd_workspace_bytes(descs, 1, hdlib.make_params(M.Params(bias_on=1))) == 0


def test_continuous_sliding_reaches_the_descriptor():
    """A moving slider (Sec. 3.1.1, method 1) is carried into the C descriptor."""
    from conftest import small2d
    from paper_0909_5215_gb300 import hd
    r = small2d()
    r.v_slide = 1e-3
    descs, _keep = hd.make_descs([r, small2d()])
    assert descs[0].v_slide == 1e-3 and descs[1].v_slide == 0.0


def test_tip_bonds_reach_the_descriptor():
    """The paper's bonded 3-D tip (Eq. 12) is carried into the C descriptor."""
    from paper_0909_5215_gb300 import hd
    from paper_0909_5215_gb300 import model as M
    r = M.paper3d()
    descs, _keep = hd.make_descs([r])
    assert descs[0].n_bonds == len(r.bonds) > 0
    assert descs[0].k_bond == 57.2 and descs[0].r_bond == 1.12
    assert [descs[0].bonds[k] for k in range(4)] == [int(v) for v in r.bonds[:2].reshape(-1)]


def test_bad_bond_index_is_refused(hdlib):
    from paper_0909_5215_gb300 import model as M
    r = M.paper2d()
    r.bonds = np.array([[0, r.n]], dtype=np.int32)
    p = M.Params(prec=1)
    descs, keep = hdlib.make_descs([r])
    assert hdlib.hd_workspace_bytes(descs, 1, hdlib.make_params(p)) == 0


def test_nose_hoover_chain_reaches_the_descriptor(hdlib):
    from conftest import small2d
    r = small2d()
    r.nhc_len, r.nhc_tau = 3, 0.7
    descs, _keep = hdlib.make_descs([r])
    assert descs[0].nhc_len == 3 and descs[0].nhc_tau == 0.7
    r.nhc_len = 9                        # longer than the library's chain
    descs, _keep = hdlib.make_descs([r])
    from paper_0909_5215_gb300 import model as M
    assert hdlib.hd_workspace_bytes(descs, 1, hdlib.make_params(M.Params())) == 0


def test_quench_statistics_split_the_three_outcomes():
    """Batch.qstats reads HD_OBS_QCONV's three codes (1 reached ftol, 2
    stopped inside the basin, 0 stopped at max_iter) into separate fractions
    and largest forces; no GPU is needed for this host logic."""
    from paper_0909_5215_gb300 import hd

    class Fake:
        pass

    f = Fake()
    ob = np.zeros((5, hd.OBS_LEN))
    ob[:, 14] = [100, 40, 40, 300, 120]        # q_iter
    ob[:, 15] = [0.009, 0.08, 0.05, 2.5, 0.004]  # q_fmax
    ob[:, 27] = [1, 2, 2, 0, 1]                # q_conv
    f.obs = lambda: ob
    f.last_flags = np.array([1, 0, 0, 0, 0], np.int32)
    q = hd.Batch.qstats(f)
    assert q["iters"] == pytest.approx(120.0) and q["iters_max"] == 300
    assert q["converged"] == pytest.approx(0.4) and q["stayed"] == pytest.approx(0.4)
    assert q["fmax"] == 0.009 and q["fmax_stay"] == 0.08 and q["fmax_unconverged"] == 2.5
    assert q["flagged"] == 1
