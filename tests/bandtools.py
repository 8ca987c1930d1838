"""Helpers for the full-size parity tests with the slope bias inside its band.

The band of Eq. 14 is not given by the paper (its parameters are inputs); for
a parity test it has to be placed where the slope actually goes, so that
DeltaV moves between 0 and DeltaV_max and the bias force is exercised.  The
band of a sampled replica is taken from an unbiased oracle pre-run of the
same steps from the same state (lattice plus its Maxwell-Boltzmann draw).
"""
import dataclasses
import math

import numpy as np


def run_band_prerun(oracle_mod, reps, p, sample, steps=100, q_lo=0.1, q_hi=0.9, skip_frac=0.2, draw=True):
    """Set sig_lo, sig_hi of every replica: sampled replicas get the q_lo..q_hi
    quantiles of sigma over an unbiased oracle pre-run (the first skip_frac of
    the steps left out); the others copy the band of the sampled replica of
    the same dimension whose size is closest on a log scale.  draw: start from
    Maxwell-Boltzmann velocities (True) or the replicas' own (None)."""
    p0 = dataclasses.replace(p, bias_on=0)
    ors = [oracle_mod.OracleReplica(reps[k], p0, draw_velocities=draw) for k in sample]
    sig = []
    for s in range(steps):
        oracle_mod.run_batch(ors, 1)
        if s >= int(skip_frac * steps):
            sig.append([o.s.sigma for o in ors])
    sig = np.array(sig)
    for c, k in enumerate(sample):
        lo, hi = np.quantile(sig[:, c], q_lo), np.quantile(sig[:, c], q_hi)
        assert hi > lo > 0.0, "degenerate sigma range in the pre-run of replica %d" % k
        reps[k].sig_lo, reps[k].sig_hi = float(lo), float(hi)
    for k, r in enumerate(reps):
        if k in sample:
            continue
        same = [j for j in sample if reps[j].dim == r.dim] or list(sample)
        j = min(same, key=lambda j: abs(math.log(reps[j].n) - math.log(r.n)))
        r.sig_lo, r.sig_hi = reps[j].sig_lo, reps[j].sig_hi


def sampled_bias_check(b, oracle_mod, reps, p, sample, steps=100, rel=1e-6, xtol=1e-4):
    """Step the GPU batch and the oracle copies of the sampled replicas `steps`
    steps from the batch's initial state; compare DeltaV, sigma and the
    boosted-clock increments.  Returns a report line per replica."""
    ob0 = b.obs()
    b.step(steps)
    ors = [oracle_mod.OracleReplica(reps[k], p, draw_velocities=True) for k in sample]
    th0 = [o.s.t_h for o in ors]
    oracle_mod.run_batch(ors, steps)
    report, fails = [], []
    for c, k in enumerate(sample):
        o = ors[c]
        ob = b.obs(k)
        dth_g, dth_o = ob["t_h"] - ob0[k, 2], o.s.t_h - th0[c]
        dtmd = ob["t_md"] - ob0[k, 1]
        boost = dth_o / dtmd
        cap = math.exp(reps[k].dvmax / reps[k].kT)
        dv_tol = rel * (abs(o.s.sigma * o.s.dVp) + abs(o.s.dV)) + 1e-12
        e_th = abs(dth_g / dth_o - 1.0)
        e_sig = abs(ob["sigma"] / o.s.sigma - 1.0)
        e_dv = abs(ob["dV"] - o.s.dV)
        e_x = float(np.abs(b.positions(k) - o.x).max())
        report.append("replica %d (dim %d, %d atoms): mean boost %.4f of cap %.2f, dV/dVmax %.3f; "
                      "rel err dt_h %.2e, sigma %.2e; |ddV| %.2e (tol %.2e); max|dx| %.1e" % (
                          k, reps[k].dim, reps[k].n, boost, cap, o.s.dV / reps[k].dvmax, e_th, e_sig, e_dv,
                          dv_tol, e_x))
        if not (e_th <= rel and e_sig <= rel and e_dv <= dv_tol and e_x < xtol):
            fails.append(k)
        if not (1.0 + 1e-9 < boost < cap * (1.0 - 1e-9)):
            fails.append(k)
    assert not fails, "\n".join(report)
    return report
