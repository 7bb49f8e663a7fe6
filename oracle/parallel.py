"""The oracle's M2M step on all host cores (oracle; test infrastructure only).

The same functions as :func:`oracle.m2m.step`, applied to fixed chunks of
CHUNK particles held by worker processes, so the oracle can be timed on every
core of a machine: per step each worker pushes its chunks, finds their cells
and kernels and sums their observables (float64, per chunk); the parent adds
the chunks' observables in chunk order (the result does not depend on the
number of workers), forms the residual, and sends the coefficients back for
the weight update.  Prior recomputes gather the energies' range and the
cell sums the same way.  Workers are started with the 'spawn' method.
"""
import multiprocessing as mp
import os

import numpy as np

CHUNK = 65536


def _worker(conn):
    from . import m2m as O
    chunks = {}
    P = None
    while True:
        msg = conn.recv()
        op = msg[0]
        if op == "init":
            _, P, parts = msg
            for cid, arrs in parts:
                chunks[cid] = dict(zip(("x", "y", "z", "vx", "vy", "vz", "w", "what"), arrs))
            conn.send(("ok",))
        elif op == "step":
            # entropy and weight sums of the current weights, push, cells,
            # observables with the current weights
            _, epoch = msg
            out = []
            for cid in sorted(chunks):
                c = chunks[cid]
                m = c["w"] > 0
                S = float(-np.sum(c["w"][m] * np.log(c["w"][m] / c["what"][m])))
                W = float(np.sum(c["w"]))
                c["x"], c["y"], c["z"], c["vx"], c["vy"], c["vz"] = O.kdk(
                    c["x"], c["y"], c["z"], c["vx"], c["vy"], c["vz"], P.potential, P.dt)
                c["kern"] = O.cells_and_kernels(c["x"], c["y"], c["z"], c["vx"], c["vy"], c["vz"], P.obs,
                                                P.incl_sin, P.incl_cos, epoch)
                out.append((cid, S, W, O.observe_from(c["kern"], c["w"], P.obs)))
            conn.send(out)
        elif op == "update":
            _, coef = msg
            for cid in sorted(chunks):
                c = chunks[cid]
                dot = O.kernel_dot(c["kern"], coef, P.obs, c["w"].shape[0])
                c["w"] = O.update_weights(c["w"], c["what"], dot, P.eps, P.mu, P.dt, P.entropy_const)
            conn.send(("ok",))
        elif op == "energy":
            out = []
            for cid in sorted(chunks):
                c = chunks[cid]
                T = c["x"].dtype.type
                E = T(0.5) * ((c["vx"] * c["vx"] + c["vy"] * c["vy"]) + c["vz"] * c["vz"]) + \
                    O.potential(c["x"], c["y"], c["z"], P.potential)
                Lz = c["x"] * c["vy"] - c["y"] * c["vx"]
                if P.prior.kind == "e_l2":          # L^2 = (Lx*Lx + Ly*Ly) + Lz*Lz, range [0, max]
                    Lx = c["y"] * c["vz"] - c["z"] * c["vy"]
                    Ly = c["z"] * c["vx"] - c["x"] * c["vz"]
                    Lz = (Lx * Lx + Ly * Ly) + Lz * Lz
                c["E"], c["Lz"] = E, Lz
                out.append((cid, float(E.min()), float(E.max()), float(np.abs(Lz).max())))
            conn.send(out)
        elif op == "cells":
            _, lo, hi, lm = msg
            out = []
            for cid in sorted(chunks):
                c = chunks[cid]
                iE = O._count_edges_le(c["E"], lo, hi, P.prior.nE)
                iL = O._count_edges_le(c["Lz"], 0.0 if P.prior.kind == "e_l2" else -lm, lm, P.prior.nL)
                c["cell"] = iE * P.prior.nL + iL
                out.append((cid, np.bincount(c["cell"], weights=c["w"], minlength=P.prior.ncells),
                            np.bincount(c["cell"], minlength=P.prior.ncells)))
            conn.send(out)
        elif op == "gather":
            _, sums, cnt = msg
            for c in chunks.values():
                c["what"] = sums[c["cell"]] / cnt[c["cell"]]
            conn.send(("ok",))
        elif op == "state":
            conn.send([(cid, {k: chunks[cid][k] for k in ("x", "y", "z", "vx", "vy", "vz", "w", "what")})
                       for cid in sorted(chunks)])
        elif op == "stop":
            conn.send(("ok",))
            return


class ParallelOracle:
    """The state of one model spread over `nproc` worker processes."""

    def __init__(self, problem, precision, nproc=None):
        from . import m2m as O
        self.O = O
        self.P = problem
        self.nproc = nproc or os.cpu_count() or 1
        st = O.init(problem, precision)
        self.Dt, self.t, self.epoch = st.Dt, 0, 0
        self.y_obs = st.y_obs
        n = st.x.shape[0]
        self.nchunks = (n + CHUNK - 1) // CHUNK
        ctx = mp.get_context("spawn")
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"            # one thread per worker process
        try:
            self.conns, self.procs = [], []
            for _ in range(min(self.nproc, self.nchunks)):
                a, b = ctx.Pipe()
                p = ctx.Process(target=_worker, args=(b,), daemon=True)
                p.start()
                self.conns.append(a)
                self.procs.append(p)
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        arrs = (st.x, st.y, st.z, st.vx, st.vy, st.vz, st.w, st.what)
        parts = [[] for _ in self.conns]
        for cid in range(self.nchunks):
            sl = slice(cid * CHUNK, min(n, (cid + 1) * CHUNK))
            parts[cid % len(self.conns)].append((cid, [a[sl].copy() for a in arrs]))
        for conn, pt in zip(self.conns, parts):
            conn.send(("init", problem, pt))
        for conn in self.conns:
            conn.recv()

    def _all(self, msg):
        for conn in self.conns:
            conn.send(msg)
        out = []
        for conn in self.conns:
            out.extend(conn.recv())
        return sorted(out, key=lambda r: r[0]) if out and isinstance(out[0], tuple) and \
            isinstance(out[0][0], (int, np.integer)) else out

    def step(self):
        """One step, as :func:`oracle.m2m.step` (returns its record)."""
        O, P = self.O, self.P
        parts = self._all(("step", self.epoch + 1))
        self.epoch += 1
        S = sum(p[1] for p in parts)
        W = sum(p[2] for p in parts)
        yv = parts[0][3].copy()
        for p in parts[1:]:
            yv = yv + p[3]
        Delta, Dt, coef, chi2, chi2_raw = O.residual(yv, P.Y, P.sigma, self.Dt, P.alpha, False)
        self._all(("update", coef))
        self.t += 1
        if P.prior.kind in ("e_lz", "e_l2") and self.t % P.prior.period == 0:
            rng = self._all(("energy",))
            lo, hi, lm = min(r[1] for r in rng), max(r[2] for r in rng), max(r[3] for r in rng)
            cs = self._all(("cells", lo, hi, lm))
            sums = cs[0][1].copy()
            cnt = cs[0][2].copy()
            for c in cs[1:]:
                sums = sums + c[1]
                cnt = cnt + c[2]
            self._all(("gather", sums, cnt))
        elif P.prior.kind not in ("flat", "e_lz", "e_l2") and self.t % P.prior.period == 0:
            raise NotImplementedError("parallel oracle: (E, L_z), (E, L^2) or flat priors only")
        self.Dt, self.y_obs = Dt, yv
        return dict(t=self.t, chi2=chi2, chi2_raw=chi2_raw, S=S, sum_w=W, F=O.merit(chi2, S, P.mu))

    def state(self):
        parts = sorted(self._all(("state",)), key=lambda r: r[0])
        return {k: np.concatenate([p[1][k] for p in parts]) for k in parts[0][1]}

    def close(self):
        for conn in self.conns:
            try:
                conn.send(("stop",))
                conn.recv()
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=5)
