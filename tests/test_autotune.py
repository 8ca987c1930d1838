"""Autotuner host logic (no GPU): choice, signature and JSON cache."""
from conftest import small2d, small3d


def test_choose_and_cache(tmp_path):
    from paper_0909_5215_gb300 import autotune, hd
    from paper_0909_5215_gb300 import model as M
    reps = [small2d(), small3d()]
    p = M.Params(prec=1)
    calls = []

    def fake(rs, params, driver, block, steps, warm):
        calls.append((driver, block))
        return {(hd.HD_DRIVER_KERNELS, 128): 2.0, (hd.HD_DRIVER_PERSISTENT, 128): 1.5}.get((driver, block), 3.0)

    cache = str(tmp_path / "tune.json")
    drv, blk, ms = autotune.tune(reps, p, cache=cache, timer=fake)
    assert (drv, blk) == (hd.HD_DRIVER_PERSISTENT, 128)
    assert len(calls) == len(autotune.CANDIDATES)
    drv2, blk2, _ = autotune.tune(reps, p, cache=cache, timer=fake)     # cached: no new timings
    assert (drv2, blk2) == (drv, blk) and len(calls) == len(autotune.CANDIDATES)
    assert autotune.signature(reps, p) != autotune.signature(reps[:1], p)
    assert autotune.choose({(1, 64): None, (1, 128): None}) == (hd.HD_DRIVER_KERNELS, 128)
