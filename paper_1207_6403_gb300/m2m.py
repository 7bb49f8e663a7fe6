"""Thin Python binding of libm2m.so (argument marshalling only).

Every entry point of ``include/m2m.h`` has a same-named function here; all
arithmetic of the M2M step runs in the library's CUDA kernels.  PyTorch
provides the device memory (particle arrays are torch tensors that the
context borrows) and the stream.  There is no fallback: if the library
cannot be built or loaded, or no GPU is present, these functions raise.
"""
import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_void_p

import numpy as np

from . import build as _build

M2M_OK = 0
ERRORS = {-1: "M2M_ERR_ARG", -2: "M2M_ERR_CUDA", -3: "M2M_ERR_NONFINITE", -4: "M2M_ERR_TIMEOUT",
          -5: "M2M_ERR_STATE", -6: "M2M_ERR_NOMEM", -7: "M2M_ERR_OVERFLOW"}
FP64, FP32C = 0, 1
POT = {"hernquist": 1, "nfw": 2, "log": 3, "sh": 4, "sh_tri": 5, "sh_full": 6}
SH_ROW = 21
TRI_ROW = 61
FULL_ROW = 101
GEOM = {"shell": 1, "annulus": 2, "grid": 3, "lut": 4}
QUANT = {"mass": 1, "vlos2": 2, "gh": 3}
PRIOR = {"flat": 0, "e_lc": 1, "e_lz": 2, "e_l2": 3}
HISTORY = 16384


class m2m_potential_desc(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("reserved", c_int32), ("p", c_double * 4)]


class m2m_obs_desc(ctypes.Structure):
    _fields_ = [("geom", c_int32), ("quant", c_int32), ("nx", c_int32), ("ny", c_int32),
                ("edges_x", POINTER(c_double)), ("edges_y", POINTER(c_double)),
                ("gh_V", POINTER(c_double)), ("gh_S", POINTER(c_double)),
                ("sigma_kernel", c_double), ("lut", POINTER(c_int32)), ("ncell", c_int32),
                ("psf_q", POINTER(c_double)), ("psf_bits", c_int32), ("psf_seed", ctypes.c_uint32)]


class m2m_prior_desc(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("nE", c_int32), ("nL", c_int32), ("period", c_int32),
                ("hernquist_GM", c_double), ("hernquist_a", c_double)]


class m2m_params(ctypes.Structure):
    _fields_ = [("eps", c_double), ("mu", c_double), ("dt", c_double), ("alpha", c_double),
                ("entropy_const", c_double), ("incl_sin", c_double), ("incl_cos", c_double)]


TK_N = 8
TIMING_KINDS = ("step_upd", "step", "residual", "update", "prior", "other", "sh", "steps")


class m2m_tuning(ctypes.Structure):
    _fields_ = [("threads", c_int32), ("pipeline", c_int32), ("us_per_step", c_double),
                ("candidates", c_int32), ("from_cache", c_int32), ("key", ctypes.c_char * 64)]


class m2m_timing(ctypes.Structure):
    _fields_ = [("launches", c_int64 * TK_N), ("ms", c_double * TK_N), ("steps", c_int64 * TK_N),
                ("kernels_total", c_int64)]


class m2m_model_desc(ctypes.Structure):
    _fields_ = [("n", c_int64), ("x", c_void_p), ("y", c_void_p), ("z", c_void_p), ("vx", c_void_p),
                ("vy", c_void_p), ("vz", c_void_p), ("w", c_void_p), ("what", c_void_p),
                ("pot", POINTER(m2m_potential_desc)), ("npot", c_int32),
                ("obs", POINTER(m2m_obs_desc)), ("nsets", c_int32),
                ("Y", POINTER(c_double)), ("sigma", POINTER(c_double)), ("eps", c_double),
                ("prior", POINTER(m2m_prior_desc))]


class m2m_record(ctypes.Structure):
    _fields_ = [("step", c_int64), ("chi2", c_double), ("chi2_raw", c_double), ("S", c_double),
                ("sum_w", c_double), ("F", c_double), ("max_abs_dt", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def library():
    """Build (if stale) and load libm2m.so; raises if that is impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        path = _build.build()
    L = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "m2m_init": (c_int32, [POINTER(P), c_int32, c_int64, P, P, P, P, P, P, P, P,
                               POINTER(m2m_potential_desc), c_int32, POINTER(m2m_obs_desc), c_int32,
                               POINTER(c_double), POINTER(c_double), POINTER(m2m_params),
                               POINTER(m2m_prior_desc), P]),
        "m2m_set_targets": (c_int32, [P, POINTER(c_double), POINTER(c_double)]),
        "m2m_potential": (c_int32, [P, POINTER(m2m_potential_desc), c_int32]),
        "m2m_observe": (c_int32, [P, c_int32]),
        "m2m_update_weights": (c_int32, [P]),
        "m2m_priors": (c_int32, [P]),
        "m2m_push": (c_int32, [P, c_int64]),
        "m2m_step": (c_int32, [P, c_int64]),
        "m2m_get_obs": (c_int32, [P, POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
        "m2m_get_record": (c_int32, [P, POINTER(m2m_record)]),
        "m2m_get_history": (c_int32, [P, c_int64, c_int64, POINTER(m2m_record)]),
        "m2m_get_cells": (c_int32, [P, P, P]),
        "m2m_nobs": (c_int64, [P]),
        "m2m_steps_taken": (c_int64, [P]),
        "m2m_set_launch": (c_int32, [P, c_int32, c_int32]),
        "m2m_set_layout": (c_int32, [P, c_int32]),
        "m2m_set_pipeline": (c_int32, [P, c_int32]),
        "m2m_set_lazy_update": (c_int32, [P, c_int32]),
        "m2m_finish_update": (c_int32, [P]),
        "m2m_get_record_async": (c_int32, [P, P]),
        "m2m_velocity_moments": (c_int32, [P, POINTER(c_double), c_int32, POINTER(c_double)]),
        "m2m_set_timing": (c_int32, [P, c_int32]),
        "m2m_set_persistent": (c_int32, [P, c_int32]),
        "m2m_set_force_cache": (c_int32, [P, c_int32]),
        "m2m_test_barrier_stall": (c_int32, [P, c_int64]),
        "m2m_get_timing": (c_int32, [P, POINTER(m2m_timing)]),
        "m2m_get_sh_table": (c_int32, [P, POINTER(c_double)]),
        "m2m_autotune": (c_int32, [P, c_int32, ctypes.c_char_p, POINTER(m2m_tuning)]),
        "m2m_observe_static": (c_int32, [c_int64, P, P, P, P, P, P, P, POINTER(m2m_obs_desc), c_int32,
                                         c_double, c_double, c_double, P, P]),
        "m2m_philox4x32_10": (c_int32, [c_int64, P, P, P]),
        "m2m_shard_init": (c_int32, [P, c_int64, c_double]),
        "m2m_shard_scatter": (c_int32, [P, c_int32, POINTER(c_int32), P, P, P]),
        "m2m_shard_residual": (c_int32, [P, P, P]),
        "m2m_shard_prior_cells": (c_int32, [P, P, P, P]),
        "m2m_shard_prior_finish": (c_int32, [P, P, P]),
        "m2m_batch_init": (c_int32, [POINTER(P), c_int32, c_int32, POINTER(m2m_model_desc),
                                     POINTER(m2m_params), P]),
        "m2m_batch_step": (c_int32, [P, c_int64]),
        "m2m_batch_autotune": (c_int32, [P, c_int32, POINTER(m2m_tuning)]),
        "m2m_batch_context": (c_int32, [P, c_int32, POINTER(P)]),
        "m2m_batch_get_records": (c_int32, [P, POINTER(m2m_record)]),
        "m2m_batch_fused": (c_int32, [P]),
        "m2m_batch_free": (c_int32, [P]),
        "m2m_last_error": (ctypes.c_char_p, [P]),
        "m2m_free": (c_int32, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


class M2MError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(rc, ctx_ptr=None):
    if rc != M2M_OK:
        msg = library().m2m_last_error(ctx_ptr)
        raise M2MError(rc, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(POINTER(c_double))


class Context:
    """A library context plus the tensors and host tables it borrows."""

    def __init__(self, ptr, tensors, keep, nobs, precision, owned=True):
        self.owned = owned
        self.ptr = ptr
        self.t = tensors          # dict name -> torch tensor (device)
        self._keep = keep
        self.nobs = nobs
        self.precision = precision

    # -- the C entry points, same names --
    def m2m_set_targets(self, Y, sigma):
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        assert Y.shape == (self.nobs,) and sigma.shape == (self.nobs,)
        self._keep["Y"], self._keep["sigma"] = Y, sigma
        _check(library().m2m_set_targets(self.ptr, _dptr(Y), _dptr(sigma)), self.ptr)

    def m2m_potential(self, comps):
        arr, n = _pot_array(comps)
        self._keep["pot"] = arr
        _check(library().m2m_potential(self.ptr, arr, n), self.ptr)

    def m2m_observe(self, mode=0):
        _check(library().m2m_observe(self.ptr, mode), self.ptr)

    def m2m_update_weights(self):
        _check(library().m2m_update_weights(self.ptr), self.ptr)

    def m2m_priors(self):
        _check(library().m2m_priors(self.ptr), self.ptr)

    def m2m_push(self, nsteps=1):
        _check(library().m2m_push(self.ptr, nsteps), self.ptr)

    def m2m_step(self, nsteps=1):
        _check(library().m2m_step(self.ptr, nsteps), self.ptr)

    def m2m_get_obs(self):
        y, D, Dt = (np.empty(self.nobs) for _ in range(3))
        _check(library().m2m_get_obs(self.ptr, _dptr(y), _dptr(D), _dptr(Dt)), self.ptr)
        return y, D, Dt

    def m2m_get_record(self):
        r = m2m_record()
        _check(library().m2m_get_record(self.ptr, byref(r)), self.ptr)
        return r.as_dict()

    def m2m_get_record_async(self, host_ptr):
        """Enqueue a copy of the last record to host_ptr (page-locked host
        memory of ctypes.sizeof(m2m_record) bytes); read it with
        m2m_record.from_address(host_ptr) once the stream has got there."""
        _check(library().m2m_get_record_async(self.ptr, c_void_p(host_ptr)), self.ptr)

    def m2m_velocity_moments(self, r2_edges):
        """(nshell, 4): sum w, sum w v_r^2, sum w v_theta^2, sum w v_phi^2 per
        shell of the r^2 edges."""
        e = np.ascontiguousarray(r2_edges, dtype=np.float64)
        out = np.zeros((len(e) - 1, 4))
        _check(library().m2m_velocity_moments(self.ptr, _dptr(e), len(e) - 1, _dptr(out)), self.ptr)
        return out

    def m2m_get_history(self, first, count):
        out = (m2m_record * count)()
        _check(library().m2m_get_history(self.ptr, first, count, out), self.ptr)
        return [r.as_dict() for r in out]

    def m2m_get_cells(self, with_prior=False):
        import torch
        n = self.t["w"].shape[0]
        nsets = self._keep["nsets"]
        oc = torch.empty(nsets * n, dtype=torch.int32, device=self.t["w"].device)
        pc = torch.empty(n, dtype=torch.int32, device=self.t["w"].device) if with_prior else None
        _check(library().m2m_get_cells(self.ptr, c_void_p(oc.data_ptr()),
                                       c_void_p(pc.data_ptr()) if pc is not None else None), self.ptr)
        torch.cuda.current_stream().synchronize()
        return oc.view(nsets, n), pc

    def m2m_nobs(self):
        return library().m2m_nobs(self.ptr)

    def m2m_steps_taken(self):
        return library().m2m_steps_taken(self.ptr)

    def m2m_set_launch(self, threads, blocks_per_sm=0):
        _check(library().m2m_set_launch(self.ptr, threads, blocks_per_sm), self.ptr)

    def m2m_set_layout(self, layout=-1):
        _check(library().m2m_set_layout(self.ptr, layout), self.ptr)

    def m2m_set_pipeline(self, enable=True):
        _check(library().m2m_set_pipeline(self.ptr, int(enable)), self.ptr)

    def m2m_set_lazy_update(self, on=True):
        _check(library().m2m_set_lazy_update(self.ptr, 1 if on else 0), self.ptr)

    def m2m_finish_update(self):
        _check(library().m2m_finish_update(self.ptr), self.ptr)

    # -- particle shards: the exchange buffers are device tensors (int64
    # totals, float64 stats and range, int64 cell sums, int32 cell counts)
    def m2m_shard_init(self, global_n, global_sum_w):
        _check(library().m2m_shard_init(self.ptr, int(global_n), float(global_sum_w)), self.ptr)

    def m2m_shard_scatter(self, push, totals, stats, rng):
        due = c_int32(0)
        _check(library().m2m_shard_scatter(self.ptr, 1 if push else 0, byref(due), c_void_p(totals.data_ptr()),
                                           c_void_p(stats.data_ptr()), c_void_p(rng.data_ptr())), self.ptr)
        return bool(due.value)

    def m2m_shard_residual(self, totals, stats):
        _check(library().m2m_shard_residual(self.ptr, c_void_p(totals.data_ptr()), c_void_p(stats.data_ptr())),
               self.ptr)

    def m2m_shard_prior_cells(self, rng, cell_sums, cell_counts):
        _check(library().m2m_shard_prior_cells(self.ptr, c_void_p(rng.data_ptr()), c_void_p(cell_sums.data_ptr()),
                                               c_void_p(cell_counts.data_ptr())), self.ptr)

    def m2m_shard_prior_finish(self, cell_sums, cell_counts):
        _check(library().m2m_shard_prior_finish(self.ptr, c_void_p(cell_sums.data_ptr()),
                                                c_void_p(cell_counts.data_ptr())), self.ptr)

    def m2m_set_force_cache(self, enable=True):
        _check(library().m2m_set_force_cache(self.ptr, 1 if enable else 0), self.ptr)

    def m2m_set_persistent(self, enable=True):
        _check(library().m2m_set_persistent(self.ptr, 1 if enable else 0), self.ptr)

    def m2m_test_barrier_stall(self, wait_ns):
        _check(library().m2m_test_barrier_stall(self.ptr, int(wait_ns)), self.ptr)

    def m2m_set_timing(self, enable):
        _check(library().m2m_set_timing(self.ptr, 1 if enable else 0), self.ptr)

    def m2m_get_timing(self):
        t = m2m_timing()
        _check(library().m2m_get_timing(self.ptr, byref(t)), self.ptr)
        return {"launches": {k: t.launches[i] for i, k in enumerate(TIMING_KINDS)},
                "ms": {k: t.ms[i] for i, k in enumerate(TIMING_KINDS)},
                "steps": {k: t.steps[i] for i, k in enumerate(TIMING_KINDS)},
                "kernels_total": t.kernels_total}

    def m2m_autotune(self, steps_per_trial=20, cache_path=None):
        """Choose launch shape and histogram privatisation by timing real
        steps (advances the model unless the cache has an entry)."""
        t = m2m_tuning()
        cp = None if cache_path is None else os.fsencode(cache_path)
        _check(library().m2m_autotune(self.ptr, int(steps_per_trial), cp, byref(t)), self.ptr)
        return {"threads": t.threads, "pipeline": t.pipeline, "us_per_step": t.us_per_step,
                "candidates": t.candidates, "from_cache": bool(t.from_cache), "key": t.key.decode()}

    def m2m_get_sh_table(self, K, triaxial=False, full=False):
        """(K, 21) node table of the spherical-harmonic component, (K, 61)
        of the triaxial one, (K, 101) of the full one (float64)."""
        import numpy as np
        out = np.zeros((K, FULL_ROW if full else TRI_ROW if triaxial else SH_ROW), dtype=np.float64)
        _check(library().m2m_get_sh_table(self.ptr, out.ctypes.data_as(POINTER(c_double))), self.ptr)
        return out

    def m2m_free(self):
        if self.ptr and self.owned:
            library().m2m_free(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.m2m_free()
        except Exception:
            pass

    # -- conveniences --
    def state(self):
        """Host copies of the particle state, a pending weight update applied
        (synchronises)."""
        import torch
        if self.ptr:
            self.m2m_finish_update()
        torch.cuda.current_stream().synchronize()
        return {k: v.cpu().numpy() for k, v in self.t.items()}


def _pot_array(comps):
    n = len(comps)
    arr = (m2m_potential_desc * max(n, 1))()
    for k, c in enumerate(comps):
        arr[k].kind = POT[c.kind]
        for j, v in enumerate(c.params):
            arr[k].p[j] = float(v)
    return arr, n


def m2m_init(precision, pos, vel, w, what, potential, obs, params, prior=None, Y=None,
             sigma=None, device="cuda:0"):
    """Create a context.

    pos, vel: (3, n) arrays (host numpy or device tensors) -- copied into new
    device tensors of the precision's dtype; w, what: (n,) float64.
    potential: list of inputs.PotentialComponent; obs: list of
    inputs.ObservableSet; params: dict(eps, mu, dt, alpha, entropy_const,
    incl_sin, incl_cos); prior: inputs.PriorSpec or None.
    """
    import torch
    lib = library()
    prec = {"fp64": FP64, "fp32c": FP32C}[precision] if isinstance(precision, str) else precision
    dt = torch.float64 if prec == FP64 else torch.float32
    dev = torch.device(device)
    t = {}
    for k, name in enumerate(("x", "y", "z")):
        t[name] = torch.as_tensor(np.asarray(pos[k]) if not torch.is_tensor(pos[k]) else pos[k]) \
            .to(device=dev, dtype=dt).contiguous().clone()
    for k, name in enumerate(("vx", "vy", "vz")):
        t[name] = torch.as_tensor(np.asarray(vel[k]) if not torch.is_tensor(vel[k]) else vel[k]) \
            .to(device=dev, dtype=dt).contiguous().clone()
    t["w"] = torch.as_tensor(w).to(device=dev, dtype=torch.float64).contiguous().clone()
    t["what"] = torch.as_tensor(what).to(device=dev, dtype=torch.float64).contiguous().clone()
    n = t["w"].shape[0]
    keep = {}
    pot_arr, npot = _pot_array(potential)
    keep["pot"] = pot_arr
    od = _obs_array(obs, keep.setdefault("obs_arrays", []))
    keep["obs"] = od
    keep["nsets"] = len(obs)
    nobs = sum(s.nobs for s in obs)
    par = m2m_params(**{k: float(params[k]) for k in
                        ("eps", "mu", "dt", "alpha", "entropy_const", "incl_sin", "incl_cos")})
    keep["par"] = par
    pd = None
    if prior is not None and prior.kind != "flat":
        pd = m2m_prior_desc(PRIOR[prior.kind], prior.nE, prior.nL, prior.period,
                            float(prior.hernquist[0]), float(prior.hernquist[1]))
        keep["prior"] = pd
    Yp = sp = None
    if Y is not None:
        keep["Y"] = np.ascontiguousarray(Y, dtype=np.float64)
        keep["sigma"] = np.ascontiguousarray(sigma, dtype=np.float64)
        Yp, sp = _dptr(keep["Y"]), _dptr(keep["sigma"])
    stream = torch.cuda.current_stream(dev).cuda_stream
    ptr = c_void_p()
    rc = lib.m2m_init(byref(ptr), prec, n,
                      *[c_void_p(t[k].data_ptr()) for k in ("x", "y", "z", "vx", "vy", "vz", "w", "what")],
                      pot_arr, npot, od, len(obs), Yp, sp, byref(par),
                      byref(pd) if pd is not None else None, c_void_p(stream))
    _check(rc, None)
    return Context(ptr, t, keep, nobs, prec)


def params_of(problem):
    """Step parameters of an inputs.Problem as the dict m2m_init takes."""
    return dict(eps=problem.eps, mu=problem.mu, dt=problem.dt, alpha=problem.alpha,
                entropy_const=problem.entropy_const, incl_sin=problem.incl_sin,
                incl_cos=problem.incl_cos)


def from_problem(problem, precision=None, device="cuda:0", targets=True):
    """m2m_init from an inputs.Problem (model particles, tables, targets)."""
    prec = precision or problem.precision
    return m2m_init(prec, problem.pos, problem.vel, problem.w0, problem.what0, problem.potential,
                    problem.obs, params_of(problem), problem.prior,
                    problem.Y if targets else None, problem.sigma if targets else None, device)


def observe_targets(problem, precision=None, device="cuda:0"):
    """Observables of the problem's target realisation, computed by the
    library (a context over the target particles, one scatter)."""
    ctx = m2m_init(precision or problem.precision, problem.target_pos, problem.target_vel,
                   problem.target_w, problem.target_w, problem.potential, problem.obs,
                   params_of(problem), None, None, None, device)
    y, _, _ = ctx.m2m_get_obs()
    ctx.m2m_free()
    return y


def m2m_observe_static(pos, vel, w, obs, incl_sin, incl_cos, weight_scale, y_out, stream=None):
    """Observables of a particle set without device allocation (see the C
    declaration): pos, vel are (x, y, z) / (vx, vy, vz) float32 device
    tensors, w a float64 device tensor, y_out a float64 device tensor of the
    observable count.  The library keeps its scratch in one fixed device
    array, so concurrent calls race; the call is enqueued on `stream` (the
    current stream by default) and returns without synchronising."""
    import torch
    lib = library()
    keep = []
    od = _obs_array(obs, keep)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    ptrs = [c_void_p(t.data_ptr()) for t in (*pos, *vel, w)]
    rc = lib.m2m_observe_static(int(w.shape[0]), *ptrs, od, len(obs), float(incl_sin), float(incl_cos),
                                float(weight_scale), c_void_p(y_out.data_ptr()), c_void_p(st))
    _check(rc, None)


def m2m_philox4x32_10(counters, keys):
    """Philox4x32-10 output words of the device routine: counters (n, 4)
    and keys (n, 2) uint32 arrays; returns (n, 4) uint32."""
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(keys, dtype=np.uint32).reshape(-1, 2)
    assert c.shape[0] == k.shape[0]
    out = np.zeros_like(c)
    _check(library().m2m_philox4x32_10(c.shape[0], c_void_p(c.ctypes.data), c_void_p(k.ctypes.data),
                                       c_void_p(out.ctypes.data)), None)
    return out


def _obs_array(obs, keep):
    od = (m2m_obs_desc * len(obs))()
    for k, s in enumerate(obs):
        ex = np.ascontiguousarray(s.edges_x, dtype=np.float64)
        keep.append(ex)
        od[k].geom, od[k].quant = GEOM[s.geom], QUANT[s.quant]
        od[k].nx, od[k].ny = len(ex) - 1, (1 if s.edges_y is None else len(s.edges_y) - 1)
        od[k].edges_x = _dptr(ex)
        if s.edges_y is not None:
            ey = np.ascontiguousarray(s.edges_y, dtype=np.float64)
            keep.append(ey)
            od[k].edges_y = _dptr(ey)
        if s.quant == "gh":
            V = np.ascontiguousarray(s.gh_V, dtype=np.float64)
            S = np.ascontiguousarray(s.gh_S, dtype=np.float64)
            keep += [V, S]
            od[k].gh_V, od[k].gh_S = _dptr(V), _dptr(S)
        od[k].sigma_kernel = float(s.sigma_kernel)
        if s.geom == "lut":
            lut = np.ascontiguousarray(s.lut, dtype=np.int32).reshape(-1)
            keep.append(lut)
            od[k].lut = lut.ctypes.data_as(POINTER(c_int32))
            od[k].ncell = int(s.ncells)
        if getattr(s, "psf_q", None) is not None:
            q = np.ascontiguousarray(s.psf_q, dtype=np.float64)
            bits = int(q.size).bit_length() - 1
            if q.size != 1 << bits:
                raise ValueError("the seeing table needs a power-of-two length")
            keep.append(q)
            od[k].psf_q, od[k].psf_bits, od[k].psf_seed = _dptr(q), bits, int(s.psf_seed) & 0xFFFFFFFF
    keep.append(od)
    return od


class Batch:
    """Several models advanced together (m2m_batch_*)."""

    def __init__(self, ptr, tensors, keep, problems, precision, stream):
        self.ptr = ptr
        self.t = tensors
        self._keep = keep
        self.problems = problems
        self.precision = precision
        self.stream = stream

    def m2m_batch_step(self, nsteps=1):
        _check(library().m2m_batch_step(self.ptr, nsteps), None)

    def m2m_batch_autotune(self, steps_per_trial=10):
        """Time 1x, 2x and 4x pass blocks on real steps and keep the fastest."""
        t = m2m_tuning()
        _check(library().m2m_batch_autotune(self.ptr, int(steps_per_trial), byref(t)), None)
        return {"us_per_step": t.us_per_step, "candidates": t.candidates, "choice": t.key.decode()}

    def m2m_batch_fused(self):
        return library().m2m_batch_fused(self.ptr)

    def m2m_batch_get_records(self):
        out = (m2m_record * len(self.problems))()
        _check(library().m2m_batch_get_records(self.ptr, out), None)
        return [r.as_dict() for r in out]

    def m2m_batch_context(self, m):
        cp = c_void_p()
        _check(library().m2m_batch_context(self.ptr, m, byref(cp)), None)
        P = self.problems[m]
        return Context(cp, self.t[m], {"nsets": len(P.obs)}, P.nobs, self.precision, owned=False)

    def m2m_batch_free(self):
        if self.ptr:
            library().m2m_batch_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.m2m_batch_free()
        except Exception:
            pass


def m2m_batch_init(precision, problems, device="cuda:0", stream=None, targets=True):
    """A batch over inputs.Problem models (their own potentials, observables,
    targets, priors and eps).  Uses a dedicated non-default stream by default
    so that the step sequence can be captured in a CUDA graph."""
    import torch
    lib = library()
    prec = {"fp64": FP64, "fp32c": FP32C}[precision] if isinstance(precision, str) else precision
    dt = torch.float64 if prec == FP64 else torch.float32
    dev = torch.device(device)
    stream = stream or torch.cuda.Stream(device=dev)
    keep, tensors = [], []
    md = (m2m_model_desc * len(problems))()
    for m, P in enumerate(problems):
        t = {}
        for k, name in enumerate(("x", "y", "z")):
            t[name] = torch.as_tensor(np.asarray(P.pos[k])).to(device=dev, dtype=dt).contiguous().clone()
        for k, name in enumerate(("vx", "vy", "vz")):
            t[name] = torch.as_tensor(np.asarray(P.vel[k])).to(device=dev, dtype=dt).contiguous().clone()
        t["w"] = torch.as_tensor(P.w0).to(device=dev, dtype=torch.float64).contiguous().clone()
        t["what"] = torch.as_tensor(P.what0).to(device=dev, dtype=torch.float64).contiguous().clone()
        tensors.append(t)
        pot, npot = _pot_array(P.potential)
        keep.append(pot)
        od = _obs_array(P.obs, keep)
        d = md[m]
        d.n = P.n
        d.x, d.y, d.z = t["x"].data_ptr(), t["y"].data_ptr(), t["z"].data_ptr()
        d.vx, d.vy, d.vz = t["vx"].data_ptr(), t["vy"].data_ptr(), t["vz"].data_ptr()
        d.w, d.what = t["w"].data_ptr(), t["what"].data_ptr()
        d.pot, d.npot = pot, npot
        d.obs, d.nsets = od, len(P.obs)
        if targets and P.Y is not None:
            Y = np.ascontiguousarray(P.Y, dtype=np.float64)
            sg = np.ascontiguousarray(P.sigma, dtype=np.float64)
            keep += [Y, sg]
            d.Y, d.sigma = _dptr(Y), _dptr(sg)
        d.eps = float(P.eps)
        if P.prior is not None and P.prior.kind != "flat":
            pd = m2m_prior_desc(PRIOR[P.prior.kind], P.prior.nE, P.prior.nL, P.prior.period,
                                float(P.prior.hernquist[0]), float(P.prior.hernquist[1]))
            keep.append(pd)
            d.prior = ctypes.pointer(pd)
    P0 = problems[0]
    par = m2m_params(eps=0.0, mu=P0.mu, dt=P0.dt, alpha=P0.alpha, entropy_const=P0.entropy_const,
                     incl_sin=P0.incl_sin, incl_cos=P0.incl_cos)
    keep += [md, par]
    torch.cuda.synchronize(dev)
    ptr = c_void_p()
    _check(lib.m2m_batch_init(byref(ptr), prec, len(problems), md, byref(par), c_void_p(stream.cuda_stream)), None)
    return Batch(ptr, tensors, keep, problems, prec, stream)
