"""The calls of hd.Batch that the sliding drivers use, on the CPU oracle.

Test infrastructure only: replicas step and quench in parallel through the
oracle's OpenMP batch calls.  adopt follows hd_quench (0 keep r_O, 1 take
the quenched positions of flagged replicas, 2 of every replica; only a
quench that reached ftol is taken), and
set_bias follows hd_set_bias (rows of DeltaV_max, sigma_L, sigma_U, m).
"""
import numpy as np

OBS_LEN = 32


class OracleBatch:
    def __init__(self, reps, params, oracle_mod):
        self.O = oracle_mod
        self.o = [oracle_mod.OracleReplica(r, params) for r in reps]
        self.xq = [o.x.copy() for o in self.o]

    def step(self, n):
        self.O.run_batch(self.o, n)

    def obs(self):
        ob = np.zeros((len(self.o), OBS_LEN))
        for k, o in enumerate(self.o):
            s = o.s
            ob[k, 0], ob[k, 1], ob[k, 2] = s.step, s.t_md, s.t_h
            ob[k, 3], ob[k, 4], ob[k, 5], ob[k, 6], ob[k, 7] = s.V, s.K, s.dV, s.sigma, s.d
            ob[k, 8], ob[k, 9], ob[k, 10], ob[k, 11] = s.FR, s.xT[0], s.xT[1], s.xT[2]
        return ob

    def quench(self, method=1, ftol=1e-4, max_iter=2000, theta=0.5, adopt=0, step_size=None):
        self.xq, _, fmax = self.O.quench_batch(self.o, method=method, ftol=ftol, max_iter=max_iter,
                                               step_size=step_size)
        flags = np.array([int(o.transition(x, theta)[0]) for o, x in zip(self.o, self.xq)], dtype=np.int32)
        for k, o in enumerate(self.o):
            # as hd_quench: only a converged quench becomes r_O
            if fmax[k] < ftol and (adopt == 2 or (adopt == 1 and flags[k])):
                o.xo[...] = self.xq[k]
                o.refresh()
        return flags

    def set_bias(self, bias):
        bias = np.asarray(bias, dtype=np.float64).reshape(len(self.o), 4)
        for o, (dvmax, lo, hi, m) in zip(self.o, bias):
            o.s.dvmax, o.s.sig_lo, o.s.sig_hi, o.s.m_exp = float(dvmax), float(lo), float(hi), int(m)
            o.refresh()

    def positions(self, k):
        return self.o[k].x.copy()

    def velocities(self, k):
        return self.o[k].v.copy()

    def qpos(self, k):
        return self.xq[k].copy()

    def ref(self, k):
        return self.o[k].xo.copy()

    def close(self):
        pass
