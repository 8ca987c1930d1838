"""Autotuner: pick the driver, tile size and pair-sweep variant of a batch
by timing them.

For a batch signature (replica sizes, dimensions, precision) each candidate
(driver in {per-phase kernels, persistent}, tile size in {64, 128, 256},
and for the split form's per-phase kernels the scalar or the packed FP32x2
pair sweep) is created on a scratch copy of the replicas, stepped `warm`
steps untimed and `steps` steps timed with CUDA events; the fastest wins.  Results are kept in
a JSON cache keyed by the signature (with the library build and the GPU
model), so a workload is tuned once per build and device.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import hd

# (driver, tile size, pair-sweep variant: 0 scalar, 1 packed FP32x2)
CANDIDATES = [(hd.HD_DRIVER_KERNELS, 128, 0), (hd.HD_DRIVER_KERNELS, 64, 0), (hd.HD_DRIVER_KERNELS, 256, 0),
              (hd.HD_DRIVER_KERNELS, 128, 1), (hd.HD_DRIVER_KERNELS, 64, 1),
              (hd.HD_DRIVER_PERSISTENT, 128, 0), (hd.HD_DRIVER_PERSISTENT, 64, 0)]
DEFAULT = (hd.HD_DRIVER_KERNELS, 128, 0)


def candidates(params):
    """The packed pair sweep exists in the split form only."""
    return [c for c in CANDIDATES if c[2] == 0 or params.prec == hd.HD_FP32_SPLIT]


def build_identity() -> str:
    """The device and the library build the timings belong to: a rebuilt
    library or another GPU model is tuned afresh."""
    from . import _build
    ident = ""
    try:
        st = os.stat(_build.OUT)
        ident = "lib%d:%d" % (st.st_size, st.st_mtime_ns)
    except OSError:
        pass
    try:
        import torch
        if torch.cuda.is_available():
            ident += ";" + torch.cuda.get_device_name()
    except ImportError:
        pass
    return ident


def signature(reps, params, ident: str = "") -> str:
    h = hashlib.sha256()
    h.update(ident.encode())
    for r in reps:
        h.update(("%d:%d:%d;" % (r.dim, r.n, int((r.role == 2).sum()))).encode())
    h.update(("prec%d bias%d rc%g skin%g" % (params.prec, params.bias_on, params.rc, params.skin)).encode())
    return h.hexdigest()[:24]


def default_cache() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "hdslide", "autotune.json")


def load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(path, table):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(timings):
    """timings: {(driver, block, pair_kernel): ms per step or None}; the
    fastest measured one."""
    ok = {k: v for k, v in timings.items() if v is not None}
    if not ok:
        return DEFAULT
    return min(ok, key=lambda k: (ok[k], k))


def time_candidate(reps, params, driver, block, steps=100, warm=20, pair_kernel=0):
    import torch
    try:
        b = hd.Batch(reps, params, driver=driver, block=block, pair_kernel=pair_kernel)
    except hd.HdError:
        return None
    if driver == hd.HD_DRIVER_PERSISTENT and b.info()["driver"] != hd.HD_DRIVER_PERSISTENT:
        b.close()
        return None
    b.step(warm)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    e1.synchronize()
    b.sync()
    ms = e0.elapsed_time(e1) / steps
    b.close()
    return ms


def tune(reps, params, cache=None, steps=100, warm=20, timer=time_candidate):
    """Return (driver, block, pair_kernel, timings) for this batch, measuring
    on a miss."""
    path = cache or default_cache()
    key = signature(reps, params, build_identity())
    table = load(path)
    if key in table and "pair_kernel" in table[key]:
        e = table[key]
        return e["driver"], e["block"], e["pair_kernel"], e.get("ms", {})
    scratch = [r.copy() for r in reps]
    timings = {c: timer(scratch, params, c[0], c[1], steps, warm, c[2]) for c in candidates(params)}
    drv, blk, pk = choose(timings)
    table[key] = {"driver": drv, "block": blk, "pair_kernel": pk,
                  "ms": {"%d/%d/%d" % k: v for k, v in timings.items()}}
    save(path, table)
    return drv, blk, pk, table[key]["ms"]
