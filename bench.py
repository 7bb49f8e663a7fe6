#!/usr/bin/env python
"""Benchmark of the M2M training step: particle-steps/s and HBM roofline.

Workload (the headline configuration): N = 4,000,000 particles in the
flattened logarithmic potential (v0=1, Rc=0.1, q=0.8) seen at 60 deg;
observables 64x64 surface-density pixels + 20x20 IFU apertures x h0..h4
(6096); moving priors on a 128x64 (E, L_z) grid every 25 steps.  Inputs are
synthetic (Philox-seeded realisations), resident in HBM when timing starts;
the particle arrays (288 MB per step of traffic) are larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload flat-log|batched|scan|sh|sh-tri|sh-full|ifu-lut|ifu-lut-seeing|recovery]

--workload batched times the 48 trial-potential models (Hernquist stars in
Hernquist + NFW halos on a 6 x 8 grid, N log-uniform in [1e5, 2e6], about
3e7 particles in all) advanced together by m2m_batch_step.
--workload scan fits one data set in the same 48 trial halos (400,000
particles each) and gathers every model's record (the potential scan).
--workload sh times the self-consistent disc + bulge (N = 8,000,000) in the
spherical-harmonic expansion of its own particles (even l <= 8, 256 nodes,
recomputed every 50 steps).
--workload sh-tri times a triaxial model (N = 4,000,000) in the triaxial
expansion of its own particles (even l <= 8, even m >= 0: 15 terms, 256
nodes, recomputed every 50 steps) with (E, L^2) moving priors;
--workload sh-full the same model rotated and shifted (no symmetry) in the
expansion with every l <= 4 and every m (25 terms, 128 nodes).
--workload ifu-lut times the flat-log galaxy observed through 300 Voronoi
bins and a long slit (apertures given by sky-pixel lookup tables);
--workload ifu-lut-seeing the same through a Gaussian PSF.
--workload recovery runs the anisotropy-recovery experiment (three initial
models of the moving-prior workload) and reports beta(r).

Prints one JSON line (rank 0).  `value` is the FP32-compensated path; the
FP64 GPU path is measured on the same box and reported under "fp64_gpu".
Under torchrun (N > 1) every rank advances its own independent model
(another seed) with no data-path collective: weak scaling.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "flat-log"
N_DEFAULT = 4_000_000
METRIC = "M2M particle-steps/s at N=4M (FP32-compensated vs FP64 GPU), % of HBM roofline"
# algorithmic bytes per particle of one steady-state step pass (FP32C):
# read x,y,z,vx,vy,vz (24) + w (8) + w_hat (8); write x..vz (24) + w (8)
BYTES_PER_PARTICLE_FP32C = 72
BYTES_PER_PARTICLE_FP64 = 120
PROFILE_JSON = os.path.join(ROOT, "profiles", "k_pass_flat_log_4M.json")


# the device code of the profiled step pass (its template, the helpers it
# inlines and the unit that instantiates it): the recorded DRAM traffic is
# used only while these are unchanged
KERNEL_SOURCES = ("m2m_device.cuh", "m2m_kernels.cuh", "m2m_steps.cuh", "m2m_steps_f32.cu", "m2m_pass_f32.cu")


def src_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1207_6403_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, n, steps_per_launch):
    """DRAM bytes (read + write) per launch of the dominant kernel from the
    committed ncu capture (profiles/k_pass_flat_log_4M.json: one entry per
    kernel, per step), or None when the capture is of other device code or
    another particle count."""
    try:
        with open(PROFILE_JSON) as f:
            prof = json.load(f)
    except Exception:
        return None
    e = prof.get("k_steps" if kernel.startswith("k_steps") else "k_pass")
    if not e or e.get("src_sha") != src_hash() or e.get("n") != n:
        return None
    return e["dram_bytes_per_step"] * steps_per_launch


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dominant(tm, pass_name):
    """(name, mean launch ms, steps per launch) of the step's dominant
    kernel from m2m_get_timing: the persistent multi-step launches where the
    model ran them, else the steady step pass (one step per launch)."""
    if tm["launches"]["steps"] > 0:
        return ("k_steps (persistent multi-step launch; per step: pending update + push + scatter + "
                "residual between grid barriers)", tm["ms"]["steps"] / tm["launches"]["steps"],
                tm["steps"]["steps"] / tm["launches"]["steps"])
    return pass_name, tm["ms"]["step_upd"] / max(1, tm["launches"]["step_upd"]), 1.0


# ------------------------------------------------------------ distributed
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        return self.reduce(x, "max")

    def sum(self, x):
        return self.reduce(x, "sum")

    def reduce(self, x, op):
        if not self.pg:
            return x
        import torch
        dev = f"cuda:{self.local}" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons in the background."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(f[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    ts += float("0." + f[0].split(".")[1]) if "." in f[0] else 0.0
                except Exception:
                    ts = None
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        inside = [r for r in rows if r[0] is not None and t0 - 0.15 <= r[0] <= t1 + 0.15]
        note = None
        if not inside:
            inside = rows
            note = "timed region shorter than the sampling interval: all samples"
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in inside for n, v in zip(names, r[3]) if v.lower() == "active"})
        out = {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
               "reasons": reasons, "samples": len(inside)}
        if note:
            out["note"] = note
        return out


# ------------------------------------------------------------ workload
def workload(n, rank=0, precision="fp32c", device="cuda:0", targets_by="gpu"):
    from paper_1207_6403_gb300 import inputs as I
    P = I.make_problem(WORKLOAD, n=n, precision=precision,
                       seed_model=5 + 1000 * rank, seed_target=6 + 1000 * rank)
    if targets_by == "gpu":
        from paper_1207_6403_gb300 import m2m as B
        Y = B.observe_targets(P, "fp32c", device)
    else:
        from oracle import m2m as O
        Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
    return P.with_targets(Y)


def config(n, world):
    return {"workload": f"{WORKLOAD}: N={n:,} particles per GPU, flattened logarithmic potential "
                        "(v0=1, Rc=0.1, q=0.8) at 60 deg, 64x64 pixels + 20x20 IFU apertures x h0..h4 "
                        "(6096 observables), (E, L_z) 128x64 moving priors every 25 steps, dt=0.01",
            "n_particles": n, "observables": 6096, "global_particles": n * world,
            "parallelism": "replicas" if world == 1 else f"{world} independent models, one per GPU",
            "l2": "particle arrays (288 MB/step) exceed the 129 MB L2; no flush needed"}


# ------------------------------------------------------------ oracle arm
def time_oracle(P, nsteps, sample_stride):
    """Oracle on a strided sample of the workload, one process; returns
    (particle-steps/s, n_sample, s)."""
    from oracle import m2m as O
    S = sample_problem(P, sample_stride)
    st = O.init(S, "fp32c")
    t0 = time.perf_counter()
    for _ in range(nsteps):
        O.step(st, S)
    dt = time.perf_counter() - t0
    return S.n * nsteps / dt, S.n, dt


def sample_problem(P, sample_stride):
    """Every sample_stride-th particle, carrying the whole model's weight (so
    the residuals and updates it computes are those of the full workload)."""
    from paper_1207_6403_gb300 import inputs as I
    sl = slice(0, None, sample_stride)
    return I.Problem(**{**P.__dict__, "n": P.pos[:, sl].shape[1], "pos": P.pos[:, sl].copy(),
                        "vel": P.vel[:, sl].copy(), "w0": P.w0[sl] * sample_stride,
                        "what0": P.what0[sl] * sample_stride})


def time_oracle_cores(P, nsteps, sample_stride=1, warmup=0, nproc=None):
    """The oracle on all host cores (oracle.parallel: worker processes started
    with 'spawn', fixed chunks of 65,536 particles); returns (particle-steps/s,
    n_sample, s, processes)."""
    from oracle.parallel import ParallelOracle
    S = P if sample_stride == 1 else sample_problem(P, sample_stride)
    po = ParallelOracle(S, "fp32c", nproc=nproc)
    try:
        for _ in range(warmup):
            po.step()
        t0 = time.perf_counter()
        for _ in range(nsteps):
            po.step()
        dt = time.perf_counter() - t0
    finally:
        po.close()
    return S.n * nsteps / dt, S.n, dt, len(po.procs)


def run_reference(args, D):
    if D.rank != 0:
        return
    P = workload(args.n, 0, targets_by="oracle")
    # the oracle on all host cores; the sample calibrated so that the whole
    # warm-up + timed run takes about two minutes
    rate, _, _, _ = time_oracle_cores(P, 1, 8)
    budget = 120.0
    per_step = budget / max(1, args.steps + args.warmup)
    n_sample = max(2000, min(args.n, int(rate * per_step)))
    stride = max(1, args.n // n_sample)
    value, ns, secs, nproc = time_oracle_cores(P, args.steps, stride, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (state f32)", "data": "synthetic", "config": config(args.n, 1),
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": nproc, "kind": "oracle",
                             "host_cpu_count": os.cpu_count(),
                             "sample": f"every {stride}th particle ({ns:,} of {args.n:,}) of the workload, "
                                       f"{args.steps} oracle steps on {nproc} processes"},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ our arm
def run_ours(args, D):
    import numpy as np
    import torch
    from paper_1207_6403_gb300 import m2m as B
    dev = f"cuda:{D.local}"
    torch.cuda.set_device(dev)
    P = workload(args.n, D.rank, device=dev)
    n = P.n
    stream = torch.cuda.current_stream()

    # ---- FP32-compensated path: the headline number (launch shape and
    # histogram privatisation autotuned on warm-up steps)
    ctx = B.from_problem(P, "fp32c", device=dev)
    tuning = ctx.m2m_autotune(max(25, args.warmup // 4), args.tune_cache)
    if args.launch != "auto":
        ctx.m2m_set_persistent(args.launch == "persistent")
        tuning["launch"] = args.launch
    ctx.m2m_step(args.warmup)
    torch.cuda.synchronize()
    ctx.m2m_get_timing()                     # reset the launch counter
    clocks = Clocks(D.local)
    clocks.start()
    D.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(stream)
    ctx.m2m_step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    D.barrier()
    clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = ctx.m2m_get_timing()["kernels_total"]
    ms_max = D.max(ms)
    value = D.world * n * args.steps / (ms_max * 1e-3)

    # ---- dominant kernel, per-launch device time (events on the launching stream)
    k_roof = min(args.steps, 2000)
    ctx.m2m_set_timing(True)
    ctx.m2m_step(k_roof)
    tm = ctx.m2m_get_timing()
    ctx.m2m_set_timing(False)
    tot_ms = sum(tm["ms"].values())
    shares = {k: round(v / tot_ms, 4) for k, v in tm["ms"].items() if v > 0}
    kernel, launch_ms, steps_per_launch = dominant(tm, "k_pass (steady-state step pass: update+push+scatter)")
    pass_ms = launch_ms / steps_per_launch
    achieved = BYTES_PER_PARTICLE_FP32C * n * steps_per_launch / (launch_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    traffic = measured_traffic(kernel, n, steps_per_launch)
    rec = ctx.m2m_get_record()
    ctx.m2m_free()

    # ---- FP64 GPU path on the same box
    k64 = max(5, min(200, args.steps // 50))
    c64 = B.from_problem(P, "fp64", device=dev)
    c64.m2m_step(2)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    c64.m2m_step(k64)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = D.max(f0.elapsed_time(f1))
    value64 = D.world * n * k64 / (ms64 * 1e-3)
    c64.m2m_free()

    # ---- equal weight accuracy: both GPU forms from the same state, 50 steps
    # (their orbits are FP32 and FP64 orbits, so particles near cell edges
    # part ways), and 50 observe + update rounds at the initial positions
    # (the weight arithmetic alone: same cells for both forms)
    ca, cb = B.from_problem(P, "fp32c", device=dev), B.from_problem(P, "fp64", device=dev)
    ca.m2m_step(50)
    cb.m2m_step(50)
    torch.cuda.synchronize()
    wrel = float(((ca.t["w"] - cb.t["w"]).abs() / cb.t["w"].abs().clamp_min(1e-300)).max().item())
    ca.m2m_free()
    cb.m2m_free()
    # (the FP64 form starts from the FP32 positions, so both compare the
    # same values against the edges; the projected coordinates are still
    # computed in each form's precision, so a particle within rounding of a
    # sky-cell edge can fall on either side: those are counted apart)
    from paper_1207_6403_gb300 import inputs as I
    P32 = I.Problem(**{**P.__dict__, "pos": P.pos.astype(np.float32).astype(np.float64),
                       "vel": P.vel.astype(np.float32).astype(np.float64)})
    ca, cb = B.from_problem(P, "fp32c", device=dev), B.from_problem(P32, "fp64", device=dev)
    for _ in range(50):
        for c in (ca, cb):
            c.m2m_observe(1)
            c.m2m_update_weights()
    torch.cuda.synchronize()
    wdiff = ((ca.t["w"] - cb.t["w"]).abs() / cb.t["w"].abs().clamp_min(1e-300))
    same = (ca.m2m_get_cells()[0] == cb.m2m_get_cells()[0]).all(dim=0)
    nd = int((~same).sum().item())
    wrel_fixed = {"max": float(wdiff.max().item()), "median": float(wdiff.median().item()),
                  "max_same_cells": float(wdiff[same].max().item()),
                  "particles_in_other_cells": nd,
                  "max_other_cells": float(wdiff[~same].max().item()) if nd else 0.0,
                  "w_change_median": float(((cb.t["w"] - torch.as_tensor(P.w0, device=dev)).abs()
                                            / torch.as_tensor(P.w0, device=dev)).median().item())}
    ca.m2m_free()
    cb.m2m_free()

    # ---- end to end through the C-ABI with host buffers: every step uploads
    # the step's targets and errors from pinned host memory and reads the
    # step's record (chi^2, S, F) back into pinned host memory; the host
    # reads step t's record while step t+1 runs (two record buffers), and
    # each call's last weight update is fused into the next call's pass
    # (lazy updates)
    import ctypes
    ce = B.from_problem(P, "fp32c", device=dev)
    ce.m2m_set_lazy_update(True)
    Yp = torch.from_numpy(P.Y).pin_memory()
    Sp = torch.from_numpy(P.sigma).pin_memory()
    Yn, Sn = Yp.numpy(), Sp.numpy()
    rsz = ctypes.sizeof(B.m2m_record)
    rbuf = torch.empty(2 * rsz, dtype=torch.uint8, pin_memory=True)
    rptr = [rbuf.data_ptr(), rbuf.data_ptr() + rsz]
    revs = [torch.cuda.Event(), torch.cuda.Event()]
    chi_host = []

    def e2e_steps(k):
        for t in range(k):
            ce.m2m_set_targets(Yn, Sn)
            ce.m2m_step(1)
            ce.m2m_get_record_async(rptr[t % 2])
            revs[t % 2].record(stream)
            if t:
                revs[(t - 1) % 2].synchronize()
                chi_host.append(B.m2m_record.from_address(rptr[(t - 1) % 2]).chi2)
        revs[(k - 1) % 2].synchronize()
        chi_host.append(B.m2m_record.from_address(rptr[(k - 1) % 2]).chi2)

    k_e2e = min(args.steps, 2000)
    e2e_steps(3)
    D.barrier()
    t0 = time.perf_counter()
    e2e_steps(k_e2e)
    ce.m2m_finish_update()          # the last step's weights, inside the timed region
    last = ce.m2m_get_record()      # synchronises; checks the kernels' error word
    t_e2e = D.max(time.perf_counter() - t0)
    assert len(chi_host) == 3 + k_e2e and chi_host[-1] == last["chi2"]
    ce.m2m_free()
    e2e = D.world * n * k_e2e / t_e2e

    cpu = None
    if D.rank == 0 and D.world == 1 and not args.no_cpu_baseline:
        # all host cores on the whole workload (10 steps), and one core on a
        # sample (every 8th particle, 3 steps)
        rate_all, ns_all, secs_all, nproc = time_oracle_cores(P, 10)
        rate, ns, secs = time_oracle(P, 3, 8)
        cpu = {"value": rate_all, "unit": "particle-steps/s", "cores": nproc, "kind": "oracle",
               "host_cpu_count": os.cpu_count(),
               "sample": f"the whole workload ({ns_all:,} particles), 10 oracle steps on {nproc} processes "
                         f"(numpy, one thread each, fixed 65,536-particle chunks; {secs_all:.1f} s)",
               "one_core": {"value": rate, "cores": 1,
                            "sample": f"every 8th particle ({ns:,} of {n:,}), 3 oracle steps ({secs:.1f} s)"}}

    if D.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": D.world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 (FP32-compensated; f64 weights)", "data": "synthetic",
                "config": config(n, D.world),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                             "bytes_per_particle": BYTES_PER_PARTICLE_FP32C, "launch_ms": launch_ms,
                             "steps_per_launch": steps_per_launch, "ms_per_step_of_kernel": pass_ms,
                             "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                             "kernel_time_shares": shares},
                "cpu_baseline": cpu,
                "e2e": {"value": e2e, "unit": "particle-steps/s",
                        "h2d_bytes_per_step": int(2 * 8 * P.nobs), "d2h_bytes_per_step": 56,
                        "how": "per step: m2m_set_targets (pinned host Y, sigma) + m2m_step(1) + "
                               "m2m_get_record_async (pinned host record, read by the host while "
                               "the next step runs), lazy weight updates"},
                "gpu_launches": int(launches),
                "clocks": clocks.summary(w0, w1),
                "tuning": tuning,
                "fp64_gpu": {"value": value64, "unit": "particle-steps/s", "steps": k64,
                             "ms_per_step": ms64 / k64,
                             "hbm_frac_at_120B": BYTES_PER_PARTICLE_FP64 * n * k64 / (ms64 * 1e-3) / 1e9 / peak},
                "fp32c_over_fp64": value / value64,
                "w_max_rel_diff_fp32c_vs_fp64_50_steps": wrel,
                "w_rel_diff_fp32c_vs_fp64_50_updates_fixed_positions": wrel_fixed,
                "last_record": {k: rec[k] for k in ("step", "chi2", "S", "sum_w", "F")}}
        print(json.dumps(line), flush=True)


def run_batched(args, D):
    import torch
    from paper_1207_6403_gb300 import inputs as I
    from paper_1207_6403_gb300 import m2m as B
    dev = f"cuda:{D.local}"
    torch.cuda.set_device(dev)
    scan = args.workload == "scan"
    if scan:
        # one data set (isotropic Hernquist stars in halo (2, 5)) fitted in
        # the 6 x 8 grid of trial halos, 400,000 particles per model
        halos = [(r, s) for r in I.HALO_MASS_RATIOS for s in I.HALO_RS]
        problems = I.make_scan(halos, (2.0, 5.0), n=400_000, n_target=2_000_000, seed=21 + 1000 * D.rank,
                               target_ra=None)
        Y = B.observe_targets(problems[0], "fp32c", dev)
        problems = [P.with_targets(Y) for P in problems]
    else:
        problems = I.make_batch(nmodels=48, seed=7 + 1000 * D.rank)
        for k, P in enumerate(problems):
            Y = B.observe_targets(P, "fp32c", dev)
            problems[k] = P.with_targets(Y)
    ntot = sum(P.n for P in problems)
    bt = B.m2m_batch_init("fp32c", problems, device=dev)
    st = bt.stream
    steps = args.steps if args.steps_given else 2000
    with torch.cuda.stream(st):
        tuning = bt.m2m_batch_autotune(max(2, args.warmup // 6))
        bt.m2m_batch_step(args.warmup)
        torch.cuda.synchronize()
        clocks = Clocks(D.local)
        clocks.start()
        D.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        e0.record(st)
        bt.m2m_batch_step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        w1 = time.time()
        clocks.stop()
    fused = bt.m2m_batch_fused()
    ms = D.max(e0.elapsed_time(e1))
    scan_out = None
    if scan:
        t0 = time.perf_counter()
        recs = bt.m2m_batch_get_records()
        gather_ms = 1e3 * (time.perf_counter() - t0)
        chi = [r["chi2"] for r in recs]
        best = min(range(len(chi)), key=chi.__getitem__)
        scan_out = {"best": {"mass_ratio": problems[best].meta["mass_ratio"], "r_s": problems[best].meta["r_s"]},
                    "true": {"mass_ratio": 2.0, "r_s": 5.0}, "chi2_min": min(chi), "chi2_max": max(chi),
                    "steps_fitted": args.warmup + steps + 2 * max(2, args.warmup // 6) * tuning["candidates"],
                    "record_gather_ms": gather_ms}
    value = D.world * ntot * steps / (ms * 1e-3)
    peak, peak_kind = peaks()
    # the step's algorithmic traffic: 72 B per particle-step over all models
    achieved = BYTES_PER_PARTICLE_FP32C * ntot * steps / (ms * 1e-3) / 1e9
    cpu = None
    if D.rank == 0 and D.world == 1 and not args.no_cpu_baseline:
        rate, ns, secs = time_oracle(problems[0], 3, 4)
        cpu = {"value": rate, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"every 4th particle of model 0 ({ns:,} of {problems[0].n:,}), 3 oracle steps "
                         f"({secs:.1f} s)"}
    if D.rank == 0:
        what = ("scan: one data set (2,000,000 isotropic Hernquist stars in halo M_h/M_* = 2, r_s/a = 5) "
                "fitted in 48 trial Hernquist + NFW potentials (6 x 8 grid), 400,000 particles each, "
                "100 shells + 60 annuli x h0..h4, flat priors" if scan else
                "batched: 48 models, Hernquist stars in Hernquist + NFW halos "
                "(M_h/M_* x r_s/a = 6 x 8 grid), N log-uniform in [1e5, 2e6], "
                "100 shells + 60 annuli x h0..h4 each, flat priors")
        line = {"metric": ("M2M particle-steps/s, potential scan over 48 trial halos (one data set)" if scan else
                           "M2M particle-steps/s, 48 batched trial-potential models"), "value": value,
                "unit": "particle-steps/s", "n_gpus": D.world, "steps": steps, "warmup": args.warmup,
                "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 (FP32-compensated; f64 weights)", "data": "synthetic",
                "config": {"workload": what,
                           "models": len(problems), "global_particles": ntot * D.world,
                           "launch": {2: "one launch per stage, CUDA graph", 1: "one launch per stage",
                                      0: "model by model"}[fused]},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None,
                             "kernel": "whole step (batched k_pass + batched residual), 72 B/particle",
                             "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
                "cpu_baseline": cpu, "clocks": clocks.summary(w0, w1), "tuning": tuning}
        if scan_out:
            line["scan"] = scan_out
        print(json.dumps(line), flush=True)
    bt.m2m_batch_free()


# workloads timed by run_single: the problem, its default size, the label of
# its bench line and the particle stride of the oracle sample
SINGLE = {
    "sh": dict(
        problem="sh-selfcons", n=8_000_000, seeds=(9, 10), stride=64,
        metric="M2M particle-steps/s, self-consistent SH potential (N=8M)",
        dtype="f32 (FP32-compensated; f64 weights, exact fixed-point SH sums)",
        kernel="k_pass (step pass: update + push in the expansion + scatter)",
        describe="sh-selfcons: N={n:,} Miyamoto-Nagai disc (a=1, b=0.2) + Hernquist bulge (a=0.3), 1:3, in "
                 "the even-l <= 8 multipole expansion of its own weighted particles on 256 log nodes in "
                 "[1e-3, 100], recomputed every 50 steps; 100 shells + 60 annuli x h0..h4, flat priors, dt=0.01"),
    "sh-tri": dict(
        problem="sh-tri", n=4_000_000, seeds=(12, 13), stride=64,
        metric="M2M particle-steps/s, self-consistent triaxial expansion (N=4M)",
        dtype="f32 (FP32-compensated; f64 weights, exact fixed-point expansion sums)",
        kernel="k_pass (step pass: update + push in the triaxial expansion + scatter)",
        describe="sh-tri: N={n:,} triaxial Hernquist-like particles (a=1, axes 1:0.8:0.6) in the even-l, "
                 "even-m >= 0, l <= 8 expansion (15 terms) of its own weighted particles on 256 log nodes in "
                 "[1e-3, 100], recomputed every 50 steps; 100 shells + 60 annuli x h0..h4, (E, L^2) 64x32 "
                 "moving priors every 25 steps, dt=0.01"),
    "sh-full": dict(
        problem="sh-full", n=4_000_000, seeds=(14, 15), stride=64,
        metric="M2M particle-steps/s, self-consistent full expansion l <= 4 (N=4M)",
        dtype="f32 (FP32-compensated; f64 weights, exact fixed-point expansion sums)",
        kernel="k_pass (step pass: update + push in the full expansion + scatter)",
        describe="sh-full: N={n:,} triaxial Hernquist-like particles (a=1, axes 1:0.8:0.6) rotated by z-y-z "
                 "Euler angles (0.5, 0.7, 0.3) and shifted by (0.05, -0.03, 0.02), in the every-l <= 4, every-m "
                 "expansion (25 terms) of its own weighted particles on 128 log nodes in [1e-3, 100], "
                 "recomputed every 50 steps; 100 shells + 60 annuli x h0..h4, (E, L^2) 64x32 moving priors "
                 "every 25 steps, dt=0.01"),
    "ifu-lut": dict(
        problem="ifu-lut", n=4_000_000, seeds=(5, 6), stride=8,
        metric="M2M particle-steps/s, IFU Voronoi bins + long slit by aperture lookup tables (N=4M)",
        dtype="f32 (FP32-compensated; f64 weights)",
        kernel="k_pass (step pass, run-time set walk: update + push + scatter through the lookup tables)",
        describe="ifu-lut: N={n:,} particles, flattened logarithmic potential (v0=1, Rc=0.1, q=0.8) at 60 deg; "
                 "64x64 pixels (mass) + 300 Voronoi bins on a 160x160 pixel table over [-2, 2]^2 x h0..h4 + "
                 "a long slit (pa 30 deg, width 0.2, 40 segments) on a 256x256 pixel table x h0..h4 "
                 "(5796 observables), (E, L_z) 128x64 moving priors every 25 steps, dt=0.01"),
    "ifu-lut-seeing": dict(
        problem="ifu-lut", kwargs=dict(seeing=0.1), n=4_000_000, seeds=(5, 6), stride=8,
        metric="M2M particle-steps/s, IFU Voronoi bins + long slit seen through a Gaussian PSF (N=4M)",
        dtype="f32 (FP32-compensated; f64 weights)",
        kernel="k_pass (step pass, run-time set walk: update + push + scatter, PSF draws per set)",
        describe="ifu-lut-seeing: the ifu-lut workload (N={n:,}) with its Voronoi and slit sets seen through a "
                 "Gaussian PSF of dispersion 0.1 per axis (4096-entry quantile table, one Philox4x32-10 draw "
                 "per particle, set and push)"),
}


def run_single(args, D):
    import torch
    from paper_1207_6403_gb300 import inputs as I
    from paper_1207_6403_gb300 import m2m as B
    W = SINGLE[args.workload]
    dev = f"cuda:{D.local}"
    torch.cuda.set_device(dev)
    n = args.n if args.n != N_DEFAULT else W["n"]
    P = I.make_problem(W["problem"], n=n, precision="fp32c", seed_model=W["seeds"][0] + 1000 * D.rank,
                       seed_target=W["seeds"][1] + 1000 * D.rank, **W.get("kwargs", {}))
    P = P.with_targets(B.observe_targets(P, "fp32c", dev))
    steps = args.steps if args.steps_given else 1000
    stream = torch.cuda.current_stream()
    ctx = B.from_problem(P, "fp32c", device=dev)
    tuning = ctx.m2m_autotune(max(25, args.warmup // 4), args.tune_cache)
    if args.launch != "auto":
        ctx.m2m_set_persistent(args.launch == "persistent")
        tuning["launch"] = args.launch
    ctx.m2m_step(args.warmup)
    torch.cuda.synchronize()
    ctx.m2m_get_timing()
    clocks = Clocks(D.local)
    clocks.start()
    D.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(stream)
    ctx.m2m_step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    D.barrier()
    clocks.stop()
    launches = ctx.m2m_get_timing()["kernels_total"]
    ms = D.max(e0.elapsed_time(e1))
    value = D.world * n * steps / (ms * 1e-3)
    k_roof = min(steps, 500)
    ctx.m2m_set_timing(True)
    ctx.m2m_step(k_roof)
    tm = ctx.m2m_get_timing()
    ctx.m2m_set_timing(False)
    tot_ms = sum(tm["ms"].values())
    shares = {k: round(v / tot_ms, 4) for k, v in tm["ms"].items() if v > 0}
    kernel, launch_ms, steps_per_launch = dominant(tm, W["kernel"])
    pass_ms = launch_ms / steps_per_launch
    peak, peak_kind = peaks()
    achieved = BYTES_PER_PARTICLE_FP32C * n * steps_per_launch / (launch_ms * 1e-3) / 1e9
    rec = ctx.m2m_get_record()
    ctx.m2m_free()
    cpu = None
    if D.rank == 0 and D.world == 1 and not args.no_cpu_baseline:
        rate, ns, secs = time_oracle(P, 3, W["stride"])
        cpu = {"value": rate, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"every {W['stride']}th particle ({ns:,} of {n:,}) of the workload, 3 oracle steps "
                         f"({secs:.1f} s, numpy, one thread)"}
    if D.rank == 0:
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": kernel,
                "bytes_per_particle": BYTES_PER_PARTICLE_FP32C, "launch_ms": launch_ms,
                "steps_per_launch": steps_per_launch, "ms_per_step_of_kernel": pass_ms,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "kernel_time_shares": shares}
        if tm["launches"]["sh"]:
            roof["sh_recompute_ms"] = tm["ms"]["sh"] / max(1, tm["launches"]["sh"] // 2)
        line = {"metric": W["metric"], "value": value,
                "unit": "particle-steps/s", "n_gpus": D.world, "steps": steps, "warmup": args.warmup,
                "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": W["dtype"], "data": "synthetic",
                "config": {"workload": W["describe"].format(n=n),
                           "n_particles": n, "global_particles": n * D.world, "observables": P.nobs,
                           "l2": f"particle arrays ({72 * n // 10**6} MB/step) exceed the 129 MB L2; "
                                 "no flush needed"},
                "roofline": roof,
                "cpu_baseline": cpu, "gpu_launches": int(launches), "clocks": clocks.summary(w0, w1),
                "tuning": tuning, "last_record": {k: rec[k] for k in ("step", "chi2", "S", "sum_w", "F")}}
        print(json.dumps(line), flush=True)


def run_recovery(args, D):
    """Anisotropy recovery from three initial models (Section 3, Fig. 1):
    the moving-prior workload at N = 1,000,000 from isotropic, radial and
    tangential initial models; particle-steps/s over the three runs and
    beta(r) before and after."""
    import numpy as np
    import torch
    from paper_1207_6403_gb300 import recovery as RC
    dev = f"cuda:{D.local}"
    torch.cuda.set_device(dev)
    n = args.n if args.n != N_DEFAULT else 1_000_000
    steps = args.steps if args.steps_given else 20000
    r_edges = np.geomspace(0.2, 5.0, 9)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out, target = RC.recovery(n, steps, r_edges, device=dev, eps_scale=args.eps_scale)
    secs = D.max(time.perf_counter() - t0)
    if D.rank == 0:
        rm = np.sqrt(r_edges[:-1] * r_edges[1:])
        prof = {k: {"initial": [round(float(v), 3) for v in b0], "final": [round(float(v), 3) for v in b1],
                    "chi2": rec["chi2"]} for k, (b0, b1, rec) in out.items()}
        spread0 = float(np.max(np.ptp(np.array([b0 for b0, _, _ in out.values()]), axis=0)))
        spread1 = float(np.max(np.ptp(np.array([b1 for _, b1, _ in out.values()]), axis=0)))
        line = {"metric": "M2M anisotropy recovery from three initial models (Section 3, Fig. 1)",
                "value": D.world * 3 * n * steps / secs, "unit": "particle-steps/s (wall clock, setup included)",
                "n_gpus": D.world, "steps": steps, "higher_is_better": True, "data": "synthetic",
                "config": {"workload": f"moving-priors: N={n:,} Hernquist stars, Osipkov-Merritt-like target "
                                       "r_a = 1; initial models isotropic, radial (r_a = 0.3), tangential "
                                       "(beta = -0.5); (E, L^2/L_c^2) 64x32 priors every 25 steps",
                           "eps_scale": args.eps_scale,
                           "shell_radii": [round(float(v), 3) for v in rm]},
                "beta_target": [round(float(v), 3) for v in target],
                "beta_target_formula": [round(float(v * v / (v * v + 1.0)), 3) for v in rm],
                "models": prof, "max_spread_initial": spread0, "max_spread_final": spread1}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", "--particles", dest="n", type=int, default=N_DEFAULT,
                    help="particles per GPU (--particles also passes through torchrun)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="flat-log", choices=["flat-log", "batched", "scan", "sh", "sh-tri", "sh-full",
                                                               "ifu-lut", "ifu-lut-seeing", "recovery"])
    ap.add_argument("--eps-scale", type=float, default=1.0,
                    help="recovery workload: multiply the adaptation rate epsilon")
    ap.add_argument("--launch", default="auto", choices=["auto", "separate", "persistent"],
                    help="FP32C step launches: the autotuner's choice, one launch per stage, or persistent "
                         "multi-step launches (for profiling one kind)")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON-lines autotuning cache: a run under a profiler reuses the plain run's choice")
    args = ap.parse_args()
    args.steps_given = any(a.startswith("--steps") for a in sys.argv[1:])
    if args.warmup < 3:
        args.warmup = 3
    D = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, D)
        elif args.workload in ("batched", "scan"):
            run_batched(args, D)
        elif args.workload == "recovery":
            run_recovery(args, D)
        elif args.workload in SINGLE:
            run_single(args, D)
        else:
            run_ours(args, D)
    finally:
        D.close()


if __name__ == "__main__":
    main()
