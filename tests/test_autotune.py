"""Autotuner host logic (no GPU): choice, signature and JSON cache."""
from conftest import small2d, small3d


def test_choose_and_cache(tmp_path):
    from paper_0909_5215_gb300 import autotune, hd
    from paper_0909_5215_gb300 import model as M
    reps = [small2d(), small3d()]
    p = M.Params(prec=1)
    calls = []

    def fake(rs, params, driver, block, steps, warm, pair_kernel=0):
        calls.append((driver, block, pair_kernel))
        return {(hd.HD_DRIVER_KERNELS, 128, 1): 2.0, (hd.HD_DRIVER_PERSISTENT, 128, 0): 1.5}.get(
            (driver, block, pair_kernel), 3.0)

    cache = str(tmp_path / "tune.json")
    drv, blk, pk, ms = autotune.tune(reps, p, cache=cache, timer=fake)
    assert (drv, blk, pk) == (hd.HD_DRIVER_PERSISTENT, 128, 0)
    assert len(calls) == len(autotune.CANDIDATES)
    drv2, blk2, pk2, _ = autotune.tune(reps, p, cache=cache, timer=fake)     # cached: no new timings
    assert (drv2, blk2, pk2) == (drv, blk, pk) and len(calls) == len(autotune.CANDIDATES)
    assert autotune.signature(reps, p) != autotune.signature(reps[:1], p)
    assert autotune.choose({(1, 64, 0): None, (1, 128, 0): None}) == (hd.HD_DRIVER_KERNELS, 128, 0)
    # the FP64 form has no packed pair sweep to try
    assert all(c[2] == 0 for c in autotune.candidates(M.Params(prec=0)))


def test_rebuilt_library_or_corrupt_cache_is_tuned_afresh(tmp_path, monkeypatch):
    from paper_0909_5215_gb300 import autotune, hd
    from paper_0909_5215_gb300 import model as M
    reps = [small2d()]
    p = M.Params(prec=1)
    calls = []

    def fake(rs, params, driver, block, steps, warm, pair_kernel=0):
        calls.append((driver, block, pair_kernel))
        return 1.0 if (driver, block, pair_kernel) == (hd.HD_DRIVER_KERNELS, 64, 1) else 2.0

    cache = str(tmp_path / "sub" / "tune.json")
    monkeypatch.setattr(autotune, "build_identity", lambda: "lib1:1|GPU A")
    assert autotune.tune(reps, p, cache=cache, timer=fake)[:3] == (hd.HD_DRIVER_KERNELS, 64, 1)
    n = len(calls)
    autotune.tune(reps, p, cache=cache, timer=fake)
    assert len(calls) == n                                  # same build: cached
    monkeypatch.setattr(autotune, "build_identity", lambda: "lib2:2|GPU A")
    autotune.tune(reps, p, cache=cache, timer=fake)
    assert len(calls) == 2 * n                              # rebuilt library: timed again
    with open(cache, "w") as f:
        f.write("{not json")
    autotune.tune(reps, p, cache=cache, timer=fake)
    assert len(calls) == 3 * n                              # unreadable cache: timed again
    # every candidate failing falls back to the per-phase kernels
    assert autotune.choose({c: None for c in autotune.CANDIDATES}) == (hd.HD_DRIVER_KERNELS, 128, 0)
