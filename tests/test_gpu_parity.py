"""GPU parity: every stage of the CUDA path against the CPU oracle on the
same seeded inputs, called through the C-ABI (thin binding).

Tolerances (each follows from the arithmetic of the path it checks):
* bin and prior-cell indices: bit-exact (float and double; the logarithm in
  the energy of the logarithmic potential is the fixed-order one of
  oracle.flog on both sides);
* positions/velocities of the Hernquist and logarithmic pushes: bit-exact;
* FP64 path: 1e-10 relative on every floating output;
* FP32-compensated path: observables |dy| <= 1e-5 * scale_j (scale_j =
  max(|y_j|, sigma_j/0.02), the bin's reference value), weights 1e-4
  relative after 1000 steps, on every element.
"""
import math

import numpy as np
import pytest

from oracle import m2m as O
from paper_1207_6403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402

_CACHE = {}


def problem(name, n, precision=None, **kw):
    key = (name, n, precision, tuple(sorted(kw.items())))
    if key not in _CACHE:
        P = I.make_problem(name, n=n, precision=precision, **kw)
        Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
        _CACHE[key] = P.with_targets(Y)
    return _CACHE[key]


def oracle_state_arrays(st):
    return dict(x=st.x, y=st.y, z=st.z, vx=st.vx, vy=st.vy, vz=st.vz, w=st.w, what=st.what)


def obs_scale(y, sigma):
    return np.maximum(np.maximum(np.abs(y), sigma / 0.02), 1e-300)


def assert_obs_close(y_gpu, y_orc, sigma, tol):
    err = np.abs(y_gpu - y_orc) / obs_scale(y_orc, sigma)
    assert err.max() <= tol, f"max scaled error {err.max():.3e} at {err.argmax()}"


# ------------------------------------------------------------------ push
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("name", ["plain-fp64", "flat-log"])
def test_push_is_bit_exact(prec, name):
    P = problem(name, 4097, prec)
    ctx = B.from_problem(P, prec)
    ctx.m2m_push(150)
    g = ctx.state()
    st = O.init(P, prec)
    s = (st.x, st.y, st.z, st.vx, st.vy, st.vz)
    for _ in range(150):
        s = O.kdk(*s, P.potential, P.dt)
    for a, k in zip(s, ("x", "y", "z", "vx", "vy", "vz")):
        assert np.array_equal(g[k], a), k
    # weights untouched by a pure push
    assert np.array_equal(g["w"], P.w0)


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-12), ("fp32c", 2e-5)])
def test_push_nfw_plus_hernquist_close(prec, rtol):
    P = problem("plain-fp64", 3001, prec)
    comps = [I.PotentialComponent("hernquist", (1.0, 1.0)), I.PotentialComponent("nfw", (0.02, 5.0))]
    P = I.Problem(**{**P.__dict__, "potential": comps})
    ctx = B.from_problem(P, prec)
    ctx.m2m_push(50)
    g = ctx.state()
    st = O.init(P, prec)
    s = (st.x, st.y, st.z, st.vx, st.vy, st.vz)
    for _ in range(50):
        s = O.kdk(*s, comps, P.dt)
    for a, k in zip(s, ("x", "y", "z", "vx", "vy", "vz")):
        np.testing.assert_allclose(g[k], a, rtol=rtol, atol=rtol * np.abs(a).max())


# ------------------------------------------------------------------ cells
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("name", ["plain-fp64", "moving-priors", "flat-log", "ifu-lut"])
def test_observable_cells_are_bit_exact(prec, name):
    P = problem(name, 20011, prec)
    ctx = B.from_problem(P, prec)
    ctx.m2m_push(7)
    oc, _ = ctx.m2m_get_cells()
    oc = oc.cpu().numpy()
    st = O.init(P, prec)
    s = (st.x, st.y, st.z, st.vx, st.vy, st.vz)
    for _ in range(7):
        s = O.kdk(*s, P.potential, P.dt)
    kern = O.cells_and_kernels(*s, P.obs, P.incl_sin, P.incl_cos)
    for k, (cell, _) in enumerate(kern):
        assert np.array_equal(oc[k], cell), f"set {k}: {np.sum(oc[k] != cell)} mismatches"


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_cells_on_edges_nan_and_out_of_range(prec):
    T = np.float64 if prec == "fp64" else np.float32
    ex = I.uniform_edges(8, -2.0, 2.0)
    ey = I.uniform_edges(4, -1.0, 1.0)
    lut = np.array([[0, 1, 1, -1, 2, 2, 3, 0]] * 2 + [[-1, 4, 4, 4, 4, 5, 5, -1]] * 2, np.int32)
    obs = [I.ObservableSet("grid", "mass", ex, ey),
           I.ObservableSet("shell", "mass", I.log_shell_edges(5, 0.1, 3.0)),
           I.ObservableSet("lut", "mass", ex, ey, lut=lut, n_apertures=6)]
    xs = np.concatenate([ex.astype(T), ex.astype(T) - np.abs(ex.astype(T)) * 1e-7,
                         np.array([np.nan, np.inf, -np.inf, 2.0, -2.0, 0.0], T)])
    n = xs.size
    ys = np.zeros(n, T)
    zs = np.zeros(n, T)
    ys[::3] = T(1.0)           # top y-edge: outside (half-open)
    ys[1::3] = T(-1.0)         # bottom y-edge: inside
    pos = np.stack([xs, ys, zs]).astype(np.float64)
    vel = np.zeros((3, n))
    w = np.full(n, 1.0 / n)
    ctx = B.m2m_init(prec, pos.astype(T), vel.astype(T), w, w, [], obs,
                     dict(eps=0, mu=0, dt=0.01, alpha=1, entropy_const=1, incl_sin=0.0, incl_cos=1.0))
    oc, _ = ctx.m2m_get_cells()
    oc = oc.cpu().numpy()
    kern = O.cells_and_kernels(xs, ys, zs, zs, zs, zs, obs, 0.0, 1.0)
    for k, (cell, _) in enumerate(kern):
        assert np.array_equal(oc[k], cell)


def _edge_neighbours(edges, T):
    """Every edge and its two neighbouring values in the state precision."""
    e = edges.astype(T)
    lo = np.nextafter(e, T(-np.inf))
    hi = np.nextafter(e, T(np.inf))
    ce = np.array([np.float32(v) if np.float32(v) >= v else np.nextafter(np.float32(v), np.float32(np.inf))
                   for v in edges], T) if T == np.float32 else e
    return np.unique(np.concatenate([e, lo, hi, ce, np.nextafter(ce, T(-np.inf))]))


@pytest.mark.parametrize("name", ["flat-log", "moving-priors", "plain-fp64"])
def test_scatter_cells_at_edge_neighbours(name):
    """The compiled scatter decides most cells from the float index guess
    alone; particles on every edge and one ulp either side of it must land
    in the same cells as the oracle's (distinct weights: a particle in the
    wrong cell moves a sum by far more than the tolerance)."""
    T = np.float32
    P = problem(name, 2000, "fp32c")
    rng = np.random.default_rng(5)
    xs, ys, zs = [], [], []
    for s in P.obs:
        if s.geom == "grid":
            vx = _edge_neighbours(s.edges_x, T)
            vy = _edge_neighbours(s.edges_y, T)
            # X = x, Y = z sin i - y cos i: with z = 0 and cos i rounding
            # to 1 or 1/2 in float, y = -Y / cos i is exact; the other axis
            # at random
            c = float(np.float32(P.incl_cos))
            assert c in (1.0, 0.5)
            ry = rng.uniform(s.edges_y[0], s.edges_y[-1], vx.size).astype(T)
            rx = rng.uniform(s.edges_x[0], s.edges_x[-1], vy.size).astype(T)
            xs += [vx, rx]
            ys += [(-ry / T(c)).astype(T), (-vy / T(c)).astype(T)]
            zs += [np.zeros(vx.size, T), np.zeros(vy.size, T)]
        else:
            # shells and annuli: edges of r^2 (R^2); a particle on the x axis
            # with x^2 landing next to each squared edge
            r = np.sqrt(_edge_neighbours(s.edges_x, np.float64))
            v = np.unique(np.concatenate([r.astype(T), np.nextafter(r.astype(T), T(0)),
                                          np.nextafter(r.astype(T), T(np.inf))]))
            xs.append(v)
            ys.append(np.zeros(v.size, T))
            zs.append(np.zeros(v.size, T))
    x, y, z = (np.concatenate(a).astype(T) for a in (xs, ys, zs))
    n = x.size
    pos = np.stack([x, y, z]).astype(np.float64)
    vel = np.stack([rng.normal(0, 0.3, n) for _ in range(3)])
    w = 1.0 + np.arange(n) / 4096.0
    ctx = B.m2m_init("fp32c", pos.astype(T), vel.astype(T), w, w, P.potential, P.obs,
                     dict(eps=0, mu=0, dt=0.01, alpha=1, entropy_const=1, incl_sin=P.incl_sin,
                          incl_cos=P.incl_cos))
    ctx.m2m_observe(0)
    yg, _, _ = ctx.m2m_get_obs()
    yo = O.observe(x, y, z, *vel.astype(T), w, P.obs, P.incl_sin, P.incl_cos)
    off = 0
    for s in P.obs:
        blk = slice(off, off + s.nobs)
        if s.quant == "mass":
            np.testing.assert_allclose(yg[blk], yo[blk], rtol=1e-12, atol=1e-9)
        else:
            np.testing.assert_allclose(yg[blk], yo[blk], rtol=1e-4, atol=1e-4)
        off += s.nobs


def _prior_cells_oracle(P, prec, nsteps):
    st = O.init(P, prec)
    s = (st.x, st.y, st.z, st.vx, st.vy, st.vz)
    for _ in range(nsteps):
        s = O.kdk(*s, P.potential, P.dt)
    return s, O.prior_cells(*s, P.prior, P.potential)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_prior_cells_hernquist_bit_exact(prec):
    P = problem("moving-priors", 30007, prec)
    ctx = B.from_problem(P, prec)
    ctx.m2m_push(3)
    _, pc = ctx.m2m_get_cells(with_prior=True)
    _, ref = _prior_cells_oracle(P, prec, 3)
    assert np.array_equal(pc.cpu().numpy(), ref)


@pytest.mark.parametrize("prec,n", [("fp32c", 200_003), ("fp64", 30_007)])
def test_prior_cells_log_potential_bit_exact(prec, n):
    """The energy's logarithm is the same fixed sequence of operations in
    the state precision on both sides (oracle.flog), so every (E, L_z) cell
    matches, at edges too."""
    P = problem("flat-log", n, prec)
    ctx = B.from_problem(P, prec)
    ctx.m2m_push(3)
    _, pc = ctx.m2m_get_cells(with_prior=True)
    _, ref = _prior_cells_oracle(P, prec, 3)
    assert np.array_equal(pc.cpu().numpy(), ref)


# --------------------------------------------------------- observe, update
@pytest.mark.parametrize("layout", [-1, 0])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32c", 1e-5)])
@pytest.mark.parametrize("name", ["plain-fp64", "moving-priors", "flat-log", "ifu-lut"])
def test_observe_residual_and_update_match(prec, tol, name, layout):
    """layout -1: the kernels compiled for the workload's observable sets;
    0: the run-time walk over the set descriptors."""
    P = problem(name, 20011, prec)
    ctx = B.from_problem(P, prec)
    ctx.m2m_set_layout(layout)
    ctx.m2m_observe(2)
    st = O.init(P, prec)
    y, D, Dt = ctx.m2m_get_obs()
    assert_obs_close(y, st.y_obs, P.sigma, tol)
    np.testing.assert_allclose(Dt, st.Dt, rtol=0, atol=tol / 0.02 * 5)   # Delta in sigma units
    np.testing.assert_allclose(D, st.Delta, rtol=0, atol=tol / 0.02 * 5)
    # one weight update with the initial Delta~
    ctx.m2m_update_weights()
    g = ctx.state()
    kern = O.cells_and_kernels(st.x, st.y, st.z, st.vx, st.vy, st.vz, P.obs, P.incl_sin, P.incl_cos)
    dot = O.kernel_dot(kern, st.coef, P.obs, P.n)
    w1 = O.update_weights(st.w, st.what, dot, P.eps, P.mu, P.dt, P.entropy_const)
    np.testing.assert_allclose(g["w"], w1, rtol=1e-12 if prec == "fp64" else 2e-7)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("name", ["moving-priors", "flat-log"])
def test_priors_match(prec, name):
    P = problem(name, 20011, prec)
    g0 = np.random.default_rng(3)
    w = P.w0 * g0.uniform(0.5, 1.5, P.n)
    P = I.Problem(**{**P.__dict__, "w0": w})
    ctx = B.from_problem(P, prec)
    ctx.m2m_priors()
    g = ctx.state()
    st = O.init(P, prec)
    cells = O.prior_cells(st.x, st.y, st.z, st.vx, st.vy, st.vz, P.prior, P.potential)
    ref = O.prior_means(st.w, cells, P.prior.ncells)
    if name == "moving-priors":
        np.testing.assert_allclose(g["what"], ref, rtol=1e-12 if prec == "fp64" else 1e-8)
    else:
        err = np.abs(g["what"] / ref - 1)
        assert np.mean(err > 1e-8) < 1e-3


# ------------------------------------------------------------ end to end
def _run_both(P, prec, nsteps):
    ctx = B.from_problem(P, prec)
    ctx.m2m_step(nsteps)
    g = ctx.state()
    y, D, Dt = ctx.m2m_get_obs()
    hist = ctx.m2m_get_history(1, nsteps)
    st = O.run(P, nsteps, precision=prec)
    return g, (y, D, Dt), hist, st


def test_plain_fp64_end_to_end_full_run():
    """The plain-method workload as stated: N=20,000, 2000 steps, FP64."""
    P = problem("plain-fp64", 20000, "fp64")
    g, (y, D, Dt), hist, st = _run_both(P, "fp64", 2000)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(g[k], getattr(st, k)), k
    np.testing.assert_allclose(g["w"], st.w, rtol=1e-10)
    assert_obs_close(y, st.y_obs, P.sigma, 1e-10)
    np.testing.assert_allclose(Dt, st.Dt, rtol=1e-10, atol=1e-10)
    for a, b in zip(hist, st.history):
        assert a["step"] == b["t"]
        for k in ("chi2", "chi2_raw", "S", "sum_w", "F"):
            assert a[k] == pytest.approx(b[k], rel=1e-10, abs=1e-12), (k, a["step"])


def test_moving_priors_fp32c_1000_steps():
    P = problem("moving-priors", 20000, "fp32c")
    g, (y, D, Dt), hist, st = _run_both(P, "fp32c", 1000)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(g[k], getattr(st, k)), k
    np.testing.assert_allclose(g["w"], st.w, rtol=1e-4)
    np.testing.assert_allclose(g["what"], st.what, rtol=1e-4)
    assert_obs_close(y, st.y_obs, P.sigma, 1e-5)
    for a, b in zip(hist[::50], st.history[::50]):
        assert a["sum_w"] == pytest.approx(b["sum_w"], rel=1e-4)
        assert a["chi2"] == pytest.approx(b["chi2"], rel=1e-4)


def _assert_fp32c_run(P, g, y, hist, st):
    """The FP32C tolerances on every element: bit-exact trajectories, weights
    and priors within 1e-4 relative, observables within 1e-5 of the bin's
    reference value; records' chi^2 and sum w within 1e-4."""
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(g[k], getattr(st, k)), k
    np.testing.assert_allclose(g["w"], st.w, rtol=1e-4)
    np.testing.assert_allclose(g["what"], st.what, rtol=1e-4)
    assert_obs_close(y, st.y_obs, P.sigma, 1e-5)
    for a, b in zip(hist[::50], st.history[::50]):
        assert a["sum_w"] == pytest.approx(b["sum_w"], rel=1e-4)
        assert a["chi2"] == pytest.approx(b["chi2"], rel=1e-4)


def test_flat_log_fp32c_1000_steps():
    """The headline configuration (flattened logarithmic potential at 60
    deg, 64x64 pixels + 20x20 IFU apertures x h0..h4, (E, L_z) priors every
    25 steps) at N = 40,000 for 1000 steps."""
    P = problem("flat-log", 40000, "fp32c")
    g, (y, D, Dt), hist, st = _run_both(P, "fp32c", 1000)
    _assert_fp32c_run(P, g, y, hist, st)


def test_ifu_lut_fp32c_1000_steps():
    """The flat-log galaxy seen through Voronoi-binned IFU apertures and a
    long slit (lookup-table apertures), 1000 steps."""
    P = problem("ifu-lut", 40000, "fp32c")
    g, (y, D, Dt), hist, st = _run_both(P, "fp32c", 1000)
    _assert_fp32c_run(P, g, y, hist, st)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_seeing_cells_are_bit_exact(prec):
    """Sets seen through a PSF: the GPU's counter-based draws and displaced
    cells equal the oracle's after any number of pushes."""
    P = problem("ifu-lut", 20011, prec, seeing=0.1)
    ctx = B.from_problem(P, prec)
    st = O.init(P, prec)
    s = (st.x, st.y, st.z, st.vx, st.vy, st.vz)
    for e in range(3):
        oc, _ = ctx.m2m_get_cells()
        oc = oc.cpu().numpy()
        kern = O.cells_and_kernels(*s, P.obs, P.incl_sin, P.incl_cos, epoch=e)
        for k, (cell, _) in enumerate(kern):
            assert np.array_equal(oc[k], cell), f"epoch {e} set {k}: {np.sum(oc[k] != cell)} mismatches"
        ctx.m2m_push(1)
        s = O.kdk(*s, P.potential, P.dt)


def test_ifu_lut_seeing_fp32c_1000_steps():
    P = problem("ifu-lut", 40000, "fp32c", seeing=0.1)
    g, (y, D, Dt), hist, st = _run_both(P, "fp32c", 1000)
    _assert_fp32c_run(P, g, y, hist, st)


def _assert_fp64_run(P, g, y, st):
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(g[k], getattr(st, k)), k
    np.testing.assert_allclose(g["w"], st.w, rtol=1e-10)
    np.testing.assert_allclose(g["what"], st.what, rtol=1e-10)
    assert_obs_close(y, st.y_obs, P.sigma, 1e-10)


def test_ifu_lut_seeing_fp64_100_steps():
    P = problem("ifu-lut", 20011, "fp64", seeing=0.1)
    g, (y, D, Dt), hist, st = _run_both(P, "fp64", 100)
    _assert_fp64_run(P, g, y, st)


def test_ifu_lut_fp64_100_steps():
    P = problem("ifu-lut", 20011, "fp64")
    g, (y, D, Dt), hist, st = _run_both(P, "fp64", 100)
    _assert_fp64_run(P, g, y, st)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("n", [1, 3, 31, 33, 4097])
def test_small_and_ragged_sizes(prec, n):
    P = problem("moving-priors", n, prec)
    P = I.Problem(**{**P.__dict__, "prior": I.PriorSpec("e_lc", 4, 4, 5, (1.0, 1.0))})
    g, (y, D, Dt), hist, st = _run_both(P, prec, 12)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(g[k], getattr(st, k)), k
    np.testing.assert_allclose(g["w"], st.w, rtol=1e-10 if prec == "fp64" else 1e-5)
    np.testing.assert_allclose(g["what"], st.what, rtol=1e-10 if prec == "fp64" else 1e-5)


def test_zero_weights_stay_zero_and_nonfinite_is_reported():
    P = problem("plain-fp64", 5000, "fp64")
    w = P.w0.copy()
    w[::7] = 0.0
    P2 = I.Problem(**{**P.__dict__, "w0": w})
    ctx = B.from_problem(P2, "fp64")
    ctx.m2m_step(20)
    g = ctx.state()
    assert np.all(g["w"][::7] == 0.0) and np.all(np.isfinite(g["w"]))
    st = O.run(P2, 20, precision="fp64")
    np.testing.assert_allclose(g["w"], st.w, rtol=1e-10)
    # a NaN weight is caught by the kernels and surfaces on the next read
    ctx.t["w"][3] = float("nan")
    ctx.m2m_step(1)
    with pytest.raises(B.M2MError) as e:
        ctx.m2m_get_record()
    assert e.value.code == -3


def test_full_size_flat_log_one_step_sampled():
    """The benchmark's workload and launch: N = 4,000,000, one step."""
    P = problem("flat-log", 4_000_000, "fp32c")
    ctx = B.from_problem(P, "fp32c")
    ctx.m2m_step(1)
    g = ctx.state()
    y, _, _ = ctx.m2m_get_obs()
    st = O.run(P, 1, precision="fp32c")
    idx = np.random.default_rng(0).choice(P.n, 20000, replace=False)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(g[k][idx], getattr(st, k)[idx]), k
    np.testing.assert_allclose(g["w"][idx], st.w[idx], rtol=1e-6)
    assert_obs_close(y, st.y_obs, P.sigma, 1e-5)
    r = ctx.m2m_get_record()
    assert r["sum_w"] == pytest.approx(st.history[-1]["sum_w"], rel=1e-6)


@pytest.mark.parametrize("prec,name", [("fp64", "moving-priors"), ("fp32c", "moving-priors"),
                                       ("fp32c", "ifu-lut")])
def test_compiled_and_generic_layouts_agree_over_a_run(prec, name):
    """Both code paths for the same sets give the same trajectory, weights
    and observables (the fixed-point histogram makes FP32C sums exact)."""
    P = problem(name, 20000, prec)
    out = []
    for layout in (-1, 0):
        ctx = B.from_problem(P, prec)
        ctx.m2m_set_layout(layout)
        ctx.m2m_step(60)
        g = ctx.state()
        y, _, _ = ctx.m2m_get_obs()
        out.append((g, y))
    (g1, y1), (g0, y0) = out
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(g1[k], g0[k])
    # the compiled layouts evaluate the Gauss-Hermite part of the update as
    # one quartic per cell, so the rounding (not the result) differs
    tol = 1e-12 if prec == "fp64" else 2e-6
    np.testing.assert_allclose(g1["w"], g0["w"], rtol=tol)
    assert_obs_close(y1, y0, P.sigma, tol)


@pytest.mark.parametrize("n,steps", [(40000, 30), (6_000_000, 3)])
def test_pipeline_and_flush_modes_are_bit_identical(n, steps):
    """The bulk-copy pipeline (chunks of 1024 particles staged through
    shared memory, ragged tail by plain loads) and both histogram flushes
    (global integer atomics, per-block slots) give the same state and
    observables as the plain pass; at 6M particles every block also
    flushes its histogram mid-pass (more than 32768 particles per block)."""
    P = problem("flat-log", n, "fp32c") if n < 10**6 else _no_target("flat-log", n)
    out = []
    for flags in (0, 1, 2, 1 | 2, 1 | 4):
        ctx = B.from_problem(P, "fp32c")
        ctx.m2m_set_pipeline(flags)
        ctx.m2m_step(steps)
        g = ctx.state()
        y, _, _ = ctx.m2m_get_obs()
        ctx.m2m_get_record()          # surfaces a recorded error, if any
        out.append((g, y))
        ctx.m2m_free()
    g0, y0 = out[0]
    for g, y in out[1:]:
        for k in ("x", "y", "z", "vx", "vy", "vz", "w", "what"):
            assert np.array_equal(g[k], g0[k]), k
        assert np.array_equal(y, y0)


def _no_target(name, n):
    P = I.make_problem(name, n=n, precision="fp32c", with_target=False)
    return P.with_targets(np.ones(P.nobs))


def test_layout_override_is_checked():
    P = problem("plain-fp64", 2000, "fp64")
    ctx = B.from_problem(P, "fp64")
    with pytest.raises(B.M2MError):
        ctx.m2m_set_layout(1)        # pixels + apertures: not this workload's sets
    ctx.m2m_set_layout(3)
    ctx.m2m_set_layout(0)
    ctx.m2m_set_layout(-1)
    # lookup-table apertures: compiled for FP32C, walked at run time in FP64
    P = problem("ifu-lut", 2000, "fp32c")
    B.from_problem(P, "fp32c").m2m_set_layout(4)
    with pytest.raises(B.M2MError):
        B.from_problem(P, "fp64").m2m_set_layout(4)
