#!/usr/bin/env python
"""Throughput of the batched hyperdynamics path on one GB300 (or N, weak scaling).

One bench step = one pass of the whole hot path over the batch: `--md-steps`
BAOAB steps of every replica (Verlet-list rebuilds as needed, LJ + H.dr pair
sweep, slope bias, Langevin update, boosted clock), then one batched FIRE
quench of every replica with the transition test (Sec. 2.3): to max |F| < 1e-2,
or to max |F| < 1e-1 for a replica whose atoms all lie within theta/2 of r_O.

Default workload: the 3-D model of 24x24x6 fcc cells plus a radius-6 tip
(14,272 atoms) at 64 slider positions spaced 0.02 sigma, bias on, split
precision (FP32 pair arithmetic, FP64 positions and sums).  Setup (untimed):
quench to seed r_O, 1000 equilibration steps, and the bias band set from the
5% and 50% quantiles of sigma over 500 unbiased steps.

Prints one JSON line.  `--impl reference` times the CPU FP64 oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s and hypertime/s: batched FP32-split vs plain FP64, one GB300"
UNIT = "atom-steps/s"
QSTEP = 0.005      # FIRE initial time step (maximum 10x)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="afm3d_hyper64")
    ap.add_argument("--prec", default="split", choices=["split", "fp64"])
    ap.add_argument("--md-steps", type=int, default=500)
    ap.add_argument("--quench-iters", type=int, default=3000)
    ap.add_argument("--quench-ftol", type=float, default=1e-2,
                    help="transition-test quench tolerance (at 1e-2 the quenched states lie within 0.014 sigma "
                         "of their minima, against the 0.5 sigma threshold); replicas that move r_O adopt only "
                         "a quench that reached it")
    ap.add_argument("--quench-stay", type=float, default=None,
                    help="early stop of a replica's quench at max|F| < this with every atom within theta/2 of "
                         "r_O (0: off; default 0.1, and off for afm3d_large32, whose r_O is seeded only to "
                         "1e-2 on a soft landscape where the early stop misses transitions)")
    ap.add_argument("--driver", default="auto", choices=["auto", "kernels", "persistent"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--pair-kernel", type=int, default=0, choices=[0, 1],
                    help="split form with --driver kernels: 0 scalar, 1 packed FP32x2 pair sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--setup-md", type=int, default=1000, help="untimed equilibration steps")
    ap.add_argument("--seed-ftol", type=float, default=0.0,
                    help="tolerance of the quench that seeds r_O (0: 1e-3 split form, 1e-6 FP64 form)")
    ap.add_argument("--profile-region", action="store_true",
                    help="cudaProfilerStart/Stop around the timed region (ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.quench_stay is None:
        args.quench_stay = 0.0 if args.workload == "afm3d_large32" else 1e-1
    return args


def reduce_over_ranks(seconds, work, dist=None, device=None):
    """Whole-job timing across ranks: the slowest rank's time and the sum of
    the work units (atom-steps, boosted time) of all ranks."""
    if dist is None:
        return float(seconds), [float(w) for w in work]
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(x) for x in work], dtype=torch.float64, device=device)
    dist.all_reduce(w)
    return float(t.item()), [float(x) for x in w.tolist()]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ workload set-up
def build_workload(name, prec, rank):
    from paper_0909_5215_gb300 import model as M
    reps, params = M.WORKLOADS[name](prec=prec)
    if rank:
        for r in reps:
            r.rep_id += 100000 * rank
    return reps, params


def prepare_batch(reps, params, driver, block, split, setup_md=1000, pair_kernel=0, seed_ftol=0.0):
    from paper_0909_5215_gb300 import autotune, hd
    tuned = None
    pk = pair_kernel
    if driver == "auto":
        drv, block, pk, ms = autotune.tune(reps, params)
        tuned = {"driver": drv, "block": block, "pair_kernel": pk, "ms_per_step": ms}
    else:
        drv = {"kernels": hd.HD_DRIVER_KERNELS, "persistent": hd.HD_DRIVER_PERSISTENT}[driver]
    b = hd.Batch(reps, params, driver=drv, block=block, pair_kernel=pk)
    b.tuned = tuned
    # seed r_O with the quenched lattice (converged: only a converged quench is
    # adopted), equilibrate, calibrate the bias band around that r_O
    b.quench(method=1, ftol=seed_ftol or (1e-3 if split else 1e-6), max_iter=20000, step_size=QSTEP, theta=1e30,
             adopt=2)
    ob = b.obs()
    b.seed_quench = {"converged": int((ob[:, 27] == 1).sum()), "of": len(reps), "iters_max": int(ob[:, 14].max()),
                     "fmax_max": float(ob[:, 15].max())}
    if setup_md > 0:
        b.step(setup_md)
    sig = []
    for _ in range(20):
        b.step(25)
        sig.append(b.obs()[:, 6])
    sig = np.array(sig)
    q05, q50 = np.quantile(sig, 0.05, axis=0), np.quantile(sig, 0.5, axis=0)
    bias = np.array([[4.0 * r.kT, q05[k], q50[k], 2.0] for k, r in enumerate(reps)])
    b.set_bias(bias)
    b.sync()
    return b, bias


def bench_step(b, md_steps, qiters, qftol, qstay):
    b.step(md_steps)
    return b.quench(method=1, ftol=qftol, max_iter=qiters, step_size=QSTEP, theta=0.5, adopt=1, ftol_stay=qstay)


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(name, seconds, threads_hint=None):
    """Time the oracle (as it stands) on a bounded sample of the workload:
    the first S replicas, m BAOAB steps, OpenMP over replicas."""
    from oracle import oracle as O
    O.build()
    reps, params = build_workload(name, 0, 0)
    nthr = O.num_threads()
    S = min(len(reps), max(1, 2 * nthr))
    sample = [O.OracleReplica(r, params) for r in reps[:S]]
    t0 = time.perf_counter()
    O.run_batch(sample, 2)
    per_step = max((time.perf_counter() - t0) / 2.0, 1e-6)
    m = max(2, int(seconds / per_step))
    th0 = sum(o.s.t_h for o in sample)
    t0 = time.perf_counter()
    O.run_batch(sample, m)
    dt = time.perf_counter() - t0
    atoms = sum(o.n for o in sample)
    th = sum(o.s.t_h for o in sample) - th0
    return {"value": atoms * m / dt, "unit": UNIT, "cores": nthr, "kind": "oracle",
            "sample": "%d of %d replicas x %d BAOAB steps (list, LJ+H.dr, bias, Langevin; quench excluded), "
                      "%.1f s" % (S, len(reps), m, dt),
            "hypertime_per_s": th / dt, "hypertime_per_s_per_replica": th / dt / S, "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    per = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(args.workload, per / 4)
    vals, ths, thr, secs, last = [], [], [], 0.0, None
    for _ in range(args.steps):
        last = oracle_sample(args.workload, per)
        vals.append(last["value"])
        ths.append(last["hypertime_per_s"])
        thr.append(last["hypertime_per_s_per_replica"])
        secs += last["seconds"]
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "hypertime_per_s": float(np.mean(ths)),
            "hypertime_per_s_per_replica": float(np.mean(thr)),
            "config": {"workload": args.workload, "sample": last["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main arm
def kernel_code_hash():
    """sha256 (16 hex digits) of the pair kernel's sources (the shared header,
    and the reduction and pair-sweep sections of the kernel file) with
    comments and blank lines removed: a capture stays valid across comment
    edits and changes elsewhere in the file."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_0909_5215_gb300", "csrc")
    kern = open(os.path.join(csrc, "hd_kernels.cu")).read()
    marks = [m.start() for m in re.finditer(r"^// -{10,} ", kern, flags=re.M)] + [len(kern)]
    parts = [open(os.path.join(csrc, "hd_internal.cuh")).read()]
    for a, b in zip(marks[:-1], marks[1:]):
        title = kern[a:kern.index("\n", a)]
        if title.rstrip().endswith(("reductions", "pair sweep")):
            parts.append(kern[a:b])
    h = hashlib.sha256()
    for text in parts:
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for line in text.splitlines():
            line = re.sub(r"//.*", "", line).strip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def committed_traffic(split):
    """DRAM bytes per launch of the pair kernel from the committed ncu summary,
    or None when the kernel sources changed since that capture."""
    import hashlib
    if not split:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", "k_pair32_afm3d_hyper64.md")).read()
        kv = dict(l.split(": ", 1) for l in text.splitlines() if l.startswith(("traffic_bytes", "kernel_code")))
        if kernel_code_hash() != kv["kernel_code_sha256_16"].strip():
            return None
        return float(kv["traffic_bytes_per_launch"])
    except Exception:
        return None


def dv_distribution(ob0, ob1):
    """Fractions of the timed MD steps (all replicas) with DeltaV = 0, inside
    the band of Eq. 14, and at DeltaV_max, from the library's counters."""
    d = ob1[:, 24:27] - ob0[:, 24:27]
    tot = float(d.sum())
    if tot <= 0:
        return None
    f = d.sum(axis=0) / tot
    per = d / np.maximum(d.sum(axis=1, keepdims=True), 1)
    return {"zero": float(f[0]), "band": float(f[1]), "max": float(f[2]),
            "replicas_mostly_at_max": int((per[:, 2] > 0.9).sum()), "replicas": int(len(d)),
            "mean_boost": float(((ob1[:, 2] - ob0[:, 2]) / np.maximum(ob1[:, 1] - ob0[:, 1], 1e-300)).mean())}


def quench_summary(qstats, args, ms, md_ms, seed):
    col = lambda k: np.array([q[k] for q in qstats])
    return {"method": "FIRE dt0 %g" % QSTEP, "ftol": args.quench_ftol, "ftol_stay": args.quench_stay,
            "max_iter": args.quench_iters, "iters_mean": float(col("iters").mean()),
            "iters_max": int(col("iters_max").max()),
            "converged_fraction": float(col("converged").mean()), "fmax_max_converged": float(col("fmax").max()),
            "stayed_fraction": float(col("stayed").mean()), "fmax_max_stayed": float(col("fmax_stay").max()),
            "unconverged_fraction": float(1.0 - col("converged").mean() - col("stayed").mean()),
            "fmax_max_unconverged": float(col("fmax_unconverged").max()),
            "flagged": int(sum(q["flagged"] for q in qstats)),
            "time_share": float(1.0 - md_ms / ms) if ms > 0 else None, "seed_quench": seed}


def mean_nnb(b):
    tot, cnt = 0, 0
    for r in range(b.n_rep):
        c = b.nbr_count(r)
        tot += int(c.sum())
        cnt += len(c)
    return tot / cnt


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    split = args.prec == "split"
    reps, params = build_workload(args.workload, 1 if split else 0, rank)
    b, bias = prepare_batch(reps, params, args.driver, args.block, split, args.setup_md, args.pair_kernel,
                            args.seed_ftol)
    natoms = sum(r.n for r in reps)
    stream = b.stream
    torch_stream = stream

    for _ in range(args.warmup):
        bench_step(b, args.md_steps, args.quench_iters, args.quench_ftol, args.quench_stay)
    b.sync()

    # ---- timed region: inputs resident in HBM; CUDA events on the library stream
    info0 = b.info()
    b.timing(2)
    b.timing(1)
    ob0 = b.obs()
    th0 = ob0[:, 2].copy()
    qstats = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    md_ms = 0.0
    if args.profile_region:
        torch.cuda.profiler.start()
    with ClockSampler(dev.index or 0) as clk:
        e0.record(torch_stream)
        for _ in range(args.steps):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(torch_stream)
            b.step(args.md_steps)
            a1.record(torch_stream)
            b.quench(method=1, ftol=args.quench_ftol, max_iter=args.quench_iters, step_size=QSTEP, theta=0.5,
                     adopt=1, ftol_stay=args.quench_stay)
            a1.synchronize()
            md_ms += a0.elapsed_time(a1)
            qstats.append(b.qstats())
        e1.record(torch_stream)
        e1.synchronize()
    torch.cuda.synchronize()
    if args.profile_region:
        torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1)
    tim = b.timing(0)
    info1 = b.info()
    ob1 = b.obs()
    th1 = ob1[:, 2]
    atom_steps = natoms * args.md_steps * args.steps
    if world > 1:
        import torch.distributed as dist
        sec, (total_steps, dth) = reduce_over_ranks(ms / 1000.0, [atom_steps, float((th1 - th0).sum())], dist, dev)
    else:
        sec, (total_steps, dth) = reduce_over_ranks(ms / 1000.0, [atom_steps, float((th1 - th0).sum())])
    value = total_steps / sec
    launches = int(info1["launches"] - info0["launches"])

    # ---- end to end through the C ABI with host buffers
    sliders = np.array([[r.slider[0], r.slider[1]] for r in reps])
    infoa = b.info()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.set_slider(sliders)                     # host -> device: slider positions
        b.step(args.md_steps)
        flags = b.quench(method=1, ftol=args.quench_ftol, max_iter=args.quench_iters, step_size=QSTEP,
                         theta=0.5, adopt=1, ftol_stay=args.quench_stay)   # device -> host: transition flags
        obs = b.obs()                             # device -> host: observables
    torch.cuda.synchronize()
    e2e_sec = time.perf_counter() - t0
    infob = b.info()
    e2e = {"value": atom_steps / e2e_sec * world, "unit": UNIT,
           "h2d_bytes_per_step": int((infob["h2d_bytes"] - infoa["h2d_bytes"]) / args.steps),
           "d2h_bytes_per_step": int((infob["d2h_bytes"] - infoa["d2h_bytes"]) / args.steps)}

    # ---- roofline of the dominant kernel (pair sweep), events in the timed region
    nnb = mean_nnb(b)
    pair_ms = tim["pair_ms"] / tim["pair_launches"] if tim["pair_launches"] else None
    # algorithmic bytes per atom-step: every unique pair's index once (half
    # list, 2 nnb), position and velocity read and written, r_O read, type
    # and role (98 B split: FP64 r, FP32 v; 122 B FP64 form); the full list
    # this kernel streams moves 4 nnb + the records and results (100 / 196 B)
    bytes_per_atom = 2.0 * nnb + (98 if split else 122)
    streamed_per_atom = 4.0 * nnb + (4 + 16 + 16 + 16 + 16 + 32 if split else 4 + 32 + 32 + 32 + 32 + 64)
    traffic = committed_traffic(split)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    if pair_ms:
        achieved = bytes_per_atom * natoms / (pair_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic,
                "kernel": ("k_pair32x2<false,false>" if b.params.pair_kernel == 1 else "k_pair32<false,false>")
                if split else "k_pair64<false,false>",
                "algorithmic_bytes_per_atom": bytes_per_atom, "mean_neighbours": nnb,
                "streamed_bytes_per_atom": streamed_per_atom,
                "streamed_frac": streamed_per_atom * natoms / (pair_ms * 1e-3) / 1e9 / hbm,
                "pair_ms_per_launch": pair_ms,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s"}
    else:
        # the persistent launch has no separate pair kernel to time
        roof = {"bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None, "traffic": None,
                "kernel": "k_persist (phases fused; no per-phase timing)", "mean_neighbours": nnb}
    phases = {k: tim[k] for k in tim if not k.startswith("reserved")}
    phases["rebuild_ms"] = tim["rebuild_prep_ms"] + tim["nlist_ms"]
    phases["rebuild_share_of_md"] = phases["rebuild_ms"] / md_ms if md_ms > 0 else None

    # ---- FP64 form on the same equilibrated window: a batch in the plain form
    # created from this batch's current state (positions, velocities, r_O,
    # clocks, bias band), timed over the same number of MD steps as one bench
    # step's MD part, list rebuilds included
    fp64 = None
    if split and not args.no_fp64_compare and rank == 0:
        from paper_0909_5215_gb300 import hd
        reps64 = []
        for k, r in enumerate(reps):
            q = r.copy()
            q.pos, q.vel, q.pos_ref = b.positions(k), b.velocities(k), b.ref(k)
            o = b.obs(k)
            q.t_h0, q.t_md0, q.step0 = o["t_h"], o["t_md"], int(o["step"])
            q.dvmax, q.sig_lo, q.sig_hi = bias[k][0], bias[k][1], bias[k][2]
            reps64.append(q)
        p64 = type(params)(**{**params.__dict__, "prec": 0})
        b64 = hd.Batch(reps64, p64, driver=hd.HD_DRIVER_KERNELS)
        n64 = args.md_steps
        b64.step(n64)           # graph capture and first replay, untimed
        b64.sync()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s64 = b64.stream
        f0.record(s64)
        b64.step(n64)
        f1.record(s64)
        f1.synchronize()
        v64 = natoms * n64 / (f0.elapsed_time(f1) / 1000.0)
        md_only = natoms * args.md_steps * args.steps / (md_ms / 1000.0)
        fp64 = {"value": v64, "unit": UNIT, "md_steps": n64, "split_md_only_over_fp64": md_only / v64,
                "window": "same equilibrated state as the split batch, %d MD steps with rebuilds, after one "
                          "untimed %d-step window" % (n64, n64)}
        b64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            c = oracle_sample(args.workload, args.cpu_seconds)
            cpu = {k: c[k] for k in ("value", "unit", "cores", "kind", "sample")}
        except Exception as ex:  # reported, not hidden
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": "failed: %s" % ex}

    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if split else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "replicas": len(reps), "atoms": natoms,
                       "md_steps_per_step": args.md_steps, "quench": "FIRE ftol %g (in-basin stop at %g), <= %d iters, theta 0.5" % (
                           args.quench_ftol, args.quench_stay, args.quench_iters),
                       "driver": {1: "kernels", 2: "persistent"}.get(b.info()["driver"], "kernels"),
                       "block": (b.tuned or {}).get("block") or args.block or 128,
                       "pair_kernel": {0: "scalar", 1: "packed FP32x2"}[(b.tuned or {}).get("pair_kernel",
                                                                                              args.pair_kernel)],
                       "autotune": b.tuned,
                       "precision": "split: FP32 pair/bias arithmetic, FP64 positions, sums, clocks" if split
                       else "FP64 throughout", "l2": "inputs larger than L2 (%.0f MB workspace)" % (
                           b.ws_bytes / 1e6), "parallelism": "replicas" if world == 1 else "replicas x%d ranks" % world},
            "hypertime_per_s": dth / sec, "hypertime_per_s_per_replica": dth / sec / len(reps),
            "md_only": {"value": atom_steps / (md_ms / 1000.0), "unit": UNIT},
            "roofline": roof, "phases_ms": phases, "fp64_form": fp64,
            "list_rebuilds_per_replica_step": float((ob1[:, 12] - ob0[:, 12]).sum()) / (len(reps) * args.md_steps *
                                                                                          args.steps),
            "quench": quench_summary(qstats, args, ms, md_ms, b.seed_quench),
            "dv_distribution": dv_distribution(ob0, ob1),
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    b.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
