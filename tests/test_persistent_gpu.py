"""The persistent single-launch driver against the per-phase kernel driver.

Both drivers run the same per-tile phases; the compiler may contract
multiply-adds differently where a phase is inlined into one kernel or the
other, so after hundreds of steps (list rebuilds included) they agree to
rounding: 1e-10 relative here, ~1e-15 measured after 50 steps.  The barrier
time-out path is exercised with the library's test hook (one CTA skips one
barrier arrival): the wait ends by itself and the host reads HD_ERR_TIMEOUT.
"""
import os

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


def _batch_inputs():
    from paper_0909_5215_gb300 import model as M
    reps = [thermalise(small2d(), amp=0.05, seed=31), thermalise(small3d(nx=6, nz=3, radius=3.0), amp=0.05, seed=32),
            thermalise(small2d(cols=20, rows=6, n_tip=13), amp=0.05, seed=33)]
    for k, r in enumerate(reps):
        r.rep_id = k
        r.dvmax, r.sig_lo, r.sig_hi = 4 * r.kT, 5.0, 40.0
    return reps


@pytest.mark.parametrize("prec", [0, 1])
def test_persistent_equals_kernel_driver(hd, prec):
    from paper_0909_5215_gb300 import model as M
    reps = _batch_inputs()
    p = M.Params(prec=prec, bias_on=1)
    a = hd.Batch(reps, p, driver=hd.HD_DRIVER_KERNELS)
    b = hd.Batch(reps, p, driver=hd.HD_DRIVER_PERSISTENT)
    assert b.info()["driver"] == hd.HD_DRIVER_PERSISTENT and b.info()["persistent_ctas"] >= len(reps)
    for n in (1, 37, 200):
        a.step(n)
        b.step(n)
    oa, ob = a.obs(), b.obs()
    assert np.allclose(oa, ob, rtol=1e-10, atol=1e-12)
    assert np.array_equal(oa[:, :2], ob[:, :2])                    # step, t_md
    nr = hd.OBS_FIELDS.index("n_rebuild")
    assert np.abs(oa[:, nr] - ob[:, nr]).max() <= 1               # a rounding-level move may flip one decision
    assert oa[:, hd.OBS_FIELDS.index("n_rebuild")].sum() > 0      # rebuilds happened inside the launch
    for k in range(len(reps)):
        assert np.abs(a.positions(k) - b.positions(k)).max() < 1e-10
        assert np.abs(a.velocities(k) - b.velocities(k)).max() < 1e-9
    a.close()
    b.close()


def test_persistent_barrier_timeout_is_reported(hd):
    from paper_0909_5215_gb300 import model as M
    r = thermalise(small3d(nx=6, nz=3, radius=3.0), amp=0.05, seed=34)
    os.environ["HD_TEST_SKIP_ARRIVE"] = "0"
    try:
        b = hd.Batch([r], M.Params(prec=1), driver=hd.HD_DRIVER_PERSISTENT)
    finally:
        del os.environ["HD_TEST_SKIP_ARRIVE"]
    assert b.info()["persistent_ctas"] >= 2
    b.step(3)
    with pytest.raises(hd.HdError) as ei:
        b.sync()
    assert ei.value.status == hd.HD_ERR_TIMEOUT
    b.close()
    # the device is still usable
    c = hd.Batch([r], M.Params(prec=1), driver=hd.HD_DRIVER_PERSISTENT)
    c.step(5)
    c.sync()
    c.close()
