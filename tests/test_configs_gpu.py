"""Full-size GPU parity on the synthetic batches, sampled, with the bias on.

* The uneven batch: 192 replicas drawn from seed 4 (2-D with 400-4,000 atoms
  and 3-D with 5,000-40,000 atoms, log-uniform sizes, T in [0.05, 0.15]),
  about 1.96M atoms, stepped by the persistent single-launch driver.
* The large 3-D batch: 64x64x10 fcc cells plus a radius-12 tip, 32 slider
  positions, about 5.36M atoms, stepped by the per-phase kernels.

For sampled replicas the lists must equal the oracle's bit for bit, the
split-form forces must be within 1e-5 RMS relative (the stated bound for the
FP32 path), and the Maxwell-Boltzmann draws within 1e-6.  Then 100 steps run
with the slope bias (Eq. 14) inside its band: each sampled replica's band is
the 10%-90% range of sigma over an unbiased oracle pre-run of the same 100
steps, so DeltaV moves between 0 and DeltaV_max during the run.  After the
100 steps, DeltaV and sigma must be within 1e-6 relative of the oracle's
(DeltaV with the sigma error pushed through Eq. 14 where the band is steep)
and the increment of the boosted clock (Eq. 3) within 1e-6 relative.

The longest 2-D strip of the uneven batch (545 sigma, 3,925 atoms) is held to
the force bound on its own: positions there sit on a fixed-point grid of
L / 2^36, fine enough for the bound at any box length.
"""
import numpy as np
import pytest

from bandtools import run_band_prerun, sampled_bias_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_5215_gb300 import _build, hd as H
    _build.build()
    return H


def rms_rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def _check_initial(b, oracle_mod, reps, p, sample, lists_only=()):
    for k in list(sample) + list(lists_only):
        o = oracle_mod.OracleReplica(reps[k], p, draw_velocities=True)
        o.nlist_cells()
        got, ref = b.rows(k), o.rows()
        bad = [i for i in range(len(ref)) if not np.array_equal(got[i], ref[i])]
        assert not bad, "replica %d: %d rows differ" % (k, len(bad))
        assert np.abs(b.velocities(k) - o.v).max() < 1e-6
        if k in sample:
            assert rms_rel(b.forces(k), o.f_lj) <= 1e-5


def test_uneven_192_in_one_persistent_launch(hd, oracle_mod):
    from paper_0909_5215_gb300 import model as M
    reps, p = M.uneven_batch(n_rep=192, seed=4, prec=1)
    ns = np.array([r.n for r in reps])
    dims = np.array([r.dim for r in reps])
    i2, i3 = np.nonzero(dims == 2)[0], np.nonzero(dims == 3)[0]
    longest2 = int(i2[np.argmax(ns[i2])])
    sample = [int(i2[np.argmin(ns[i2])]), longest2, int(i3[np.argmin(ns[i3])]), int(i3[np.argmax(ns[i3])])]
    run_band_prerun(oracle_mod, reps, p, sample, steps=100)
    b = hd.Batch(reps, p, driver=hd.HD_DRIVER_PERSISTENT)
    assert b.info()["driver"] == hd.HD_DRIVER_PERSISTENT
    _check_initial(b, oracle_mod, reps, p, sample)
    report = sampled_bias_check(b, oracle_mod, reps, p, sample, steps=100)
    print("\n".join(report))
    b.close()


def test_split_forces_on_longest_2d_strip(hd, oracle_mod):
    """The 545-sigma strip: forces at the lattice and after 200 thermal steps
    within the 1e-5 RMS bound of the FP32 path."""
    from paper_0909_5215_gb300 import model as M
    r = M.afm2d(n_cols=486, eps=M.PAPER_EPS_2D)
    p = M.Params(prec=1, bias_on=0)
    b = hd.Batch([r], p)
    o = oracle_mod.OracleReplica(r, p, draw_velocities=True)
    o.nlist_cells()
    try:
        assert rms_rel(b.forces(0), o.f_lj) <= 1e-5
        b.step(200)
        o.run(200)
        assert rms_rel(b.forces(0), o.f_lj) <= 1e-5
        assert np.abs(b.positions(0) - o.x).max() < 1e-4
    finally:
        b.close()


def test_large_3d_batch_sampled(hd, oracle_mod):
    from paper_0909_5215_gb300 import model as M
    reps, p = M.afm3d_large(n_rep=32, prec=1)
    sample = [0, 17, 31]
    run_band_prerun(oracle_mod, reps, p, [17], steps=60)
    for r in reps:
        r.sig_lo, r.sig_hi = reps[17].sig_lo, reps[17].sig_hi
    b = hd.Batch(reps, p, driver=hd.HD_DRIVER_KERNELS)
    _check_initial(b, oracle_mod, reps, p, [0, 31])
    report = sampled_bias_check(b, oracle_mod, reps, p, sample, steps=60)
    print("\n".join(report))
    b.close()
