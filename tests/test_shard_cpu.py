"""The particle-sharded step on CPU (gloo, world size 2): the driver in
paper_1207_6403_gb300/shard.py, its exchange over torch.distributed, and
the exactness of the decomposition.

Each rank holds a stand-in for a shard context (FakeShard, below) that
takes the library's step sequence -- pending update, push, scatter into
integer totals at the whole model's fixed-point scale, residual from the
summed totals, prior cells from the summed range and cell sums -- with the
oracle's functions on its slice of the particles.  Two gloo ranks, each
with half the particles, end with exactly the weights and priors of one
rank holding all of them (integer sums do not depend on how the particles
are split), and the observables agree to the float64 rounding of the
fixed-point scale."""
import json
import math
import os
import socket

import numpy as np
import pytest

from oracle import m2m as O
from paper_1207_6403_gb300 import inputs as I
from paper_1207_6403_gb300 import shard as SH

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NSTEPS = 27           # a prior recompute after step 25


def _problem():
    P = I.make_problem("flat-log", n=6000, precision="fp32c")
    Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
    return P.with_targets(Y)


class FakeShard:
    """The shard calls of the C-ABI on one slice of particles, with the
    oracle's arithmetic and integer (fixed-point) totals."""

    def __init__(self, P, lo, hi):
        self.P = P
        st = O.init(P, "fp32c")
        self.x, self.y, self.z = (a[lo:hi].copy() for a in (st.x, st.y, st.z))
        self.vx, self.vy, self.vz = (a[lo:hi].copy() for a in (st.vx, st.vy, st.vz))
        self.w, self.what = st.w[lo:hi].copy(), st.what[lo:hi].copy()
        e2 = math.ceil(math.log2(float(np.sum(P.w0))))
        self.sh = 25 + math.ceil(math.log2(P.n)) - e2
        self.cell_shift = 60 - e2
        self.pending, self.t, self.epoch, self.Dt, self.coef = False, 0, 0, None, None

    def _update(self):
        dot = O.kernel_dot(self.kern, self.coef, self.P.obs, self.w.shape[0])
        self.w = O.update_weights(self.w, self.what, dot, self.P.eps, self.P.mu, self.P.dt, self.P.entropy_const)
        self.pending = False

    def m2m_shard_scatter(self, push, totals, stats, rng):
        P = self.P
        due = bool(push) and P.prior.kind != "flat" and (self.t + 1) % P.prior.period == 0
        if self.pending:
            self._update()
        stats[0], stats[1] = O.entropy(self.w, self.what), float(np.sum(self.w))
        if push:
            self.x, self.y, self.z, self.vx, self.vy, self.vz = O.kdk(
                self.x, self.y, self.z, self.vx, self.vy, self.vz, P.potential, P.dt)
            self.epoch += 1
        self.kern = O.cells_and_kernels(self.x, self.y, self.z, self.vx, self.vy, self.vz, P.obs,
                                        P.incl_sin, P.incl_cos, self.epoch)
        tot = np.zeros(P.nobs, dtype=np.int64)
        off = 0
        for (cell, K), s in zip(self.kern, P.obs):
            m = cell >= 0
            for k in range(s.nmom):
                q = np.rint(np.ldexp(self.w[m] * K[m, k], self.sh)).astype(np.int64)
                np.add.at(tot, off + cell[m] * s.nmom + k, q)
            off += s.nobs
        totals[:] = torch.from_numpy(tot)
        if due:
            T = self.x.dtype.type
            E = T(0.5) * ((self.vx * self.vx + self.vy * self.vy) + self.vz * self.vz) + \
                O.potential(self.x, self.y, self.z, P.potential)
            Lz = self.x * self.vy - self.y * self.vx
            self.E, self.Lz = E, Lz
            rng[0], rng[1], rng[2] = float(E.min()), -float(E.max()), -float(np.abs(Lz).max())
        self.push, self.due = bool(push), due
        return due

    def m2m_shard_residual(self, totals, stats):
        P = self.P
        yv = totals.numpy().astype(np.float64) * math.ldexp(1.0, -self.sh)
        Delta, Dt, coef, chi2, chi2_raw = O.residual(yv, P.Y, P.sigma, self.Dt, P.alpha, not self.push)
        self.y_obs, self.Dt, self.coef = yv, Dt, coef
        self.pending = self.push
        if self.push:
            self.t += 1
        totals.zero_()

    def m2m_shard_prior_cells(self, rng, cell_sums, cell_counts):
        P = self.P
        if self.pending:
            self._update()
        lo, hi, lm = float(rng[0]), -float(rng[1]), -float(rng[2])
        iE = O._count_edges_le(self.E, lo, hi, P.prior.nE)
        iL = O._count_edges_le(self.Lz, -lm, lm, P.prior.nL)
        self.cells = iE * P.prior.nL + iL
        q = np.rint(np.ldexp(self.w, self.cell_shift)).astype(np.int64)
        cell_sums[:] = torch.from_numpy(_int_bincount(self.cells, q, P.prior.ncells))
        cell_counts[:] = torch.from_numpy(np.bincount(self.cells, minlength=P.prior.ncells).astype(np.int32))

    def m2m_shard_prior_finish(self, cell_sums, cell_counts):
        s = cell_sums.numpy().astype(np.float64) * math.ldexp(1.0, -self.cell_shift)
        c = cell_counts.numpy().astype(np.float64)
        self.what = s[self.cells] / c[self.cells]


def _int_bincount(cells, q, n):
    out = np.zeros(n, dtype=np.int64)
    np.add.at(out, cells, q)
    return out


def _buffers(P):
    nc = SH.ncells_of(P.prior)
    return SH.ShardBuffers(torch.zeros(P.nobs, dtype=torch.int64), torch.zeros(2, dtype=torch.float64),
                           torch.zeros(3, dtype=torch.float64), torch.zeros(nc, dtype=torch.int64),
                           torch.zeros(nc, dtype=torch.int32))


def _run(shards, reduce):
    SH.start(shards, reduce)
    for _ in range(NSTEPS):
        SH.step(shards, reduce)


def _rank_main(rank, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    P = _problem()
    lo, hi = SH.shard_bounds(P.n, 2, rank)
    f = FakeShard(P, lo, hi)
    _run([(f, _buffers(P))], SH.DistReduce(dist))
    dist.destroy_process_group()
    np.savez(f"{out}.{rank}.npz", w=f.w, what=f.what, x=f.x, y=f.y_obs)


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_bounds_cover_the_particles_once():
    for n in (1, 7, 4_000_000, 4_000_001):
        for world in (1, 2, 3, 8):
            b = [SH.shard_bounds(n, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            sizes = [h - l for l, h in b]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_equal_one_rank_bit_for_bit(tmp_path):
    mp = torch.multiprocessing.get_context("spawn")
    port = _port()
    out = str(tmp_path / "shard")
    procs = [mp.Process(target=_rank_main, args=(r, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    r0, r1 = np.load(f"{out}.0.npz"), np.load(f"{out}.1.npz")
    # one rank holding every particle
    P = _problem()
    f = FakeShard(P, 0, P.n)
    _run([(f, _buffers(P))], SH.LocalReduce())
    assert np.array_equal(np.concatenate([r0["w"], r1["w"]]), f.w)
    assert np.array_equal(np.concatenate([r0["what"], r1["what"]]), f.what)
    assert np.array_equal(np.concatenate([r0["x"], r1["x"]]), f.x)
    assert np.array_equal(r0["y"], f.y_obs) and np.array_equal(r1["y"], f.y_obs)


def test_fake_shard_follows_the_oracle():
    """The stand-in takes the oracle's steps (its integer totals round each
    term at 2^-25 of the average weight)."""
    P = _problem()
    f = FakeShard(P, 0, P.n)
    b = _buffers(P)
    SH.start([(f, b)], SH.LocalReduce())
    st = O.init(P, "fp32c")
    for _ in range(3):
        SH.step([(f, b)], SH.LocalReduce())
        O.step(st, P)
    f._update()
    assert np.array_equal(f.x, st.x)
    np.testing.assert_allclose(f.w, st.w, rtol=1e-7)
    np.testing.assert_allclose(f.y_obs, st.y_obs, rtol=0, atol=1e-7 * np.abs(st.y_obs).max())
