"""hd_nlist_static: the neighbour-list build on caller buffers, no allocation.

For callers that must not let a library allocate device memory (a program
that budgets all GPU memory itself, or a loop that cannot afford an
allocation's latency or failure).  Its rows must equal the oracle's list
(every j != i with FP64 minimum-image r^2 below (rc + skin)^2, ascending j)
and the existing path's (hd_create + hd_read of the list), bit for bit, on
two calls in a row: the second call reuses the shared file-scope scratch left
by the first.  After a first call, further calls change neither the device's
free memory nor PyTorch's allocator.  Named to be collected last.
"""
import numpy as np
import pytest

from conftest import small2d, small3d, thermalise

pytestmark = pytest.mark.gpu


def test_static_list_matches_oracle_and_existing_entry_point(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_5215_gb300 import _build, hd
    from paper_0909_5215_gb300 import model as M
    _build.build()
    p = M.Params(prec=1)
    reps = [thermalise(small2d(), amp=0.06, seed=21), thermalise(small3d(nx=6, nz=3, radius=3.0), amp=0.06, seed=22)]
    stream = torch.cuda.Stream()
    for r in reps:
        b = hd.Batch([r], p)
        ref = b.nbr(0)
        maxnb = b.maxnb
        b.close()
        o = oracle_mod.OracleReplica(r, p, maxnb=maxnb)
        o.nlist_brute()
        pos = torch.tensor(r.pos, dtype=torch.float64, device="cuda")
        for call in range(2):
            nbr = torch.full((r.n, maxnb), 7, dtype=torch.int32, device="cuda")
            nnb = torch.zeros(r.n, dtype=torch.int32, device="cuda")
            st = hd.hd_nlist_static(pos.data_ptr(), r.n, r.box, r.periodic, p.rc + p.skin, maxnb, nbr.data_ptr(),
                                    nnb.data_ptr(), stream.cuda_stream)
            assert st == hd.HD_OK, hd.STATUS_NAMES.get(st, st)
            got = nbr.cpu().numpy()
            cnt = nnb.cpu().numpy()
            assert np.array_equal(got, ref), "call %d: rows differ from hd_create's" % call
            assert np.array_equal(cnt, o.nnb), "call %d: row lengths differ from the oracle's" % call
            rows = [got[i, : cnt[i]] for i in range(r.n)]
            assert all(np.array_equal(g, e) for g, e in zip(rows, o.rows())), "call %d: rows differ" % call


def test_static_list_allocates_nothing():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_5215_gb300 import _build, hd
    _build.build()
    r = thermalise(small3d(nx=6, nz=3, radius=3.0), amp=0.06, seed=23)
    pos = torch.tensor(r.pos, dtype=torch.float64, device="cuda")
    nbr = torch.zeros((r.n, 112), dtype=torch.int32, device="cuda")
    nnb = torch.zeros(r.n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    args = (pos.data_ptr(), r.n, r.box, r.periodic, 2.8, 112, nbr.data_ptr(), nnb.data_ptr(), stream.cuda_stream)
    assert hd.hd_nlist_static(*args) == hd.HD_OK          # first call: module and scratch committed
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(5):
        assert hd.hd_nlist_static(*args) == hd.HD_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_static_list_rejects_oversize_input():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_5215_gb300 import hd
    pos = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    nbr = torch.zeros((4, 8), dtype=torch.int32, device="cuda")
    nnb = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert hd.hd_nlist_static(pos.data_ptr(), 70000, (10.0, 10.0, 0.0), (1, 1, 0), 2.8, 8, nbr.data_ptr(),
                              nnb.data_ptr(), 0) == hd.HD_ERR_ARG
    assert hd.hd_nlist_static(pos.data_ptr(), 4, (10.0, 10.0, 0.0), (1, 1, 0), 2.8, 500, nbr.data_ptr(),
                              nnb.data_ptr(), 0) == hd.HD_ERR_ARG
