"""The particle-sharded step on one GPU: a model split into two shard
contexts (halves of its particles, exchange buffers summed on the device
by the driver's local reduction) against the same model in one context:
positions, weights, priors, observables, Delta and Delta~ bit for bit after
60 steps (two prior recomputes); the records' sums to rounding.  Between
processes the exchange is a torch.distributed all-reduce of the same
buffers: two processes, each with one shard context on this GPU, reduce
over gloo (the exchange runs between launches on the host, so no kernel
of one process waits on the other's)."""
import os
import socket

import numpy as np
import pytest

from oracle import m2m as O
from paper_1207_6403_gb300 import inputs as I
from paper_1207_6403_gb300 import shard as SH

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402


@pytest.mark.parametrize("name,n,world", [("flat-log", 60_011, 2), ("moving-priors", 40_009, 3),
                                          ("ifu-lut", 30_007, 2)])
def test_shards_take_the_steps_of_one_context(name, n, world):
    P = I.make_problem(name, n=n, precision="fp32c")
    P = P.with_targets(O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos))
    shards = [SH.make_shard(P, world, r) for r in range(world)]
    red = SH.LocalReduce()
    SH.start(shards, red)
    for _ in range(60):
        SH.step(shards, red)
    one = B.from_problem(P, "fp32c")
    one.m2m_step(60)
    g1 = one.state()
    y1, D1, Dt1 = one.m2m_get_obs()
    h1 = one.m2m_get_history(1, 60)
    gs = [c.state() for c, _ in shards]
    for k in ("x", "y", "z", "vx", "vy", "vz", "w", "what"):
        assert np.array_equal(np.concatenate([g[k] for g in gs]), g1[k]), k
    for c, _ in shards:
        y, D, Dt = c.m2m_get_obs()
        assert np.array_equal(y, y1) and np.array_equal(D, D1) and np.array_equal(Dt, Dt1)
        h = c.m2m_get_history(1, 60)
        for a, b in zip(h, h1):
            assert a["step"] == b["step"]
            assert a["chi2"] == pytest.approx(b["chi2"], rel=1e-12)
            assert a["sum_w"] == pytest.approx(b["sum_w"], rel=1e-6)
    for c, _ in shards:
        c.m2m_free()
    one.m2m_free()


def test_shard_calls_check_their_state():
    P = I.make_problem("flat-log", n=5000, precision="fp32c")
    P = P.with_targets(O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos))
    ctx = B.from_problem(P, "fp32c")
    bufs = SH.ShardBuffers.alloc(ctx.nobs, SH.ncells_of(P.prior), "cuda:0")
    with pytest.raises(B.M2MError):         # not a shard yet
        ctx.m2m_shard_scatter(True, bufs.totals, bufs.stats, bufs.rng)
    ctx.m2m_shard_init(P.n, 1.0)
    with pytest.raises(B.M2MError):         # a shard steps through the shard calls
        ctx.m2m_step(1)
    with pytest.raises(B.M2MError):         # no prior recompute is due
        ctx.m2m_shard_prior_finish(bufs.cell_sums, bufs.cell_counts)
    ctx.m2m_free()


def _port():
    with socket.socket() as s_:
        s_.bind(("127.0.0.1", 0))
        return s_.getsockname()[1]


def _rank_main(rank, port, out, nsteps):
    import torch as T
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    T.cuda.set_device(0)
    P = I.make_problem("flat-log", n=50_003, precision="fp32c")
    P = P.with_targets(O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos))
    ctx, bufs = SH.make_shard(P, 2, rank, device="cuda:0")
    red = SH.DistReduce(dist)
    SH.start([(ctx, bufs)], red)
    for _ in range(nsteps):
        SH.step([(ctx, bufs)], red)
    g = ctx.state()
    y, D, Dt = ctx.m2m_get_obs()
    np.savez(f"{out}.{rank}.npz", yobs=y, Dt=Dt, **{k: g[k] for k in ("x", "y", "z", "vx", "vy", "vz", "w", "what")})
    ctx.m2m_free()
    dist.destroy_process_group()


def test_two_processes_with_shard_contexts_equal_one_context(tmp_path):
    nsteps = 30
    mp = torch.multiprocessing.get_context("spawn")
    port = _port()
    out = str(tmp_path / "shard")
    procs = [mp.Process(target=_rank_main, args=(r, port, out, nsteps)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
        assert p.exitcode == 0
    r0, r1 = np.load(f"{out}.0.npz"), np.load(f"{out}.1.npz")
    P = I.make_problem("flat-log", n=50_003, precision="fp32c")
    P = P.with_targets(O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos))
    one = B.from_problem(P, "fp32c")
    one.m2m_step(nsteps)
    g1 = one.state()
    y1, _, Dt1 = one.m2m_get_obs()
    for k in ("x", "y", "z", "vx", "vy", "vz", "w", "what"):
        assert np.array_equal(np.concatenate([r0[k], r1[k]]), g1[k]), k
    for r in (r0, r1):
        assert np.array_equal(r["yobs"], y1) and np.array_equal(r["Dt"], Dt1)
    one.m2m_free()

