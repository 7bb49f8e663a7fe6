"""GPU parity of the full expansion (potential kind 'sh_full': every l <= 4
and every m, cosine and sine harmonics) on a rotated and shifted triaxial
model with no symmetry: node tables against the oracle's node sums,
pushes, the recompute schedule, the force kept between pushes, the
weights and observables on the GPU's own orbits, and the full-size
workload on samples.  Tolerances as for the axisymmetric and triaxial
expansions: tables to 1e-12 (FP64) / 2e-6 (FP32C) of the monopole scale,
every one of the 25 terms held to that absolute bound; trajectories of
orbits that stay outside r = 0.05 to 1e-10 relative (FP64) / 2e-5 of their
range (FP32C); weights and observables on the GPU's orbits to 1e-10 /
1e-4 relative and 1e-10 / 1e-5 of the observable's scale.
"""
import numpy as np
import pytest

from oracle import m2m as O
from paper_1207_6403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402

NT = 25
_CACHE = {}


def full_problem(n, prec, K=64, period=5, seed=14, targets=True):
    key = (n, prec, K, period, seed, targets)
    if key not in _CACHE:
        P = I.make_problem("sh-full", n=n, precision=prec, seed_model=seed, seed_target=seed + 1,
                           with_target=targets)
        P.potential = [I.PotentialComponent("sh_full", (K, 1e-3, 100.0, period))]
        P.prior = I.PriorSpec("flat")
        if targets:
            Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
            P = P.with_targets(Y)
        else:
            P = P.with_targets(np.ones(P.nobs))
        _CACHE[key] = P
    return _CACHE[key]


def split_table(T):
    return T[:, 0:25].T, T[:, 25:50].T, T[:, 50:75].T, T[:, 75:100].T, T[:, 100]


def assert_tables_close(T, ref, tol):
    F, SF, D, SD, rk = split_table(T)
    Fo, Do, rn = ref
    assert Fo.shape == (NT, len(rn))
    np.testing.assert_array_equal(rk, rn if tol < 1e-9 else rn.astype(np.float32))
    sF, sD = np.abs(Fo[0]).max(), np.abs(Do[0]).max()
    assert np.abs(F - Fo).max() <= tol * sF, (np.abs(F - Fo).max() / sF,
                                              np.unravel_index(np.abs(F - Fo).argmax(), F.shape))
    assert np.abs(D - Do).max() <= tol * sD, (np.abs(D - Do).max() / sD,
                                              np.unravel_index(np.abs(D - Do).argmax(), D.shape))
    h = np.diff(rn)
    np.testing.assert_allclose(SF[:, :-1] * h, np.diff(Fo, axis=1), rtol=0, atol=4 * tol * sF)
    np.testing.assert_allclose(SD[:, :-1] * h, np.diff(Do, axis=1), rtol=0, atol=4 * tol * sD)
    assert np.all(SF[:, -1] == 0) and np.all(SD[:, -1] == 0)


def resolved(rmin_traj):
    keep = rmin_traj > 0.05
    assert keep.mean() > 0.9
    return keep


def assert_positions_close(g, s, keep, prec, keys=("x", "y", "z", "vx", "vy", "vz")):
    for a, k in zip(s, keys):
        if prec == "fp64":
            np.testing.assert_allclose(g[k][keep], a[keep], rtol=1e-10, atol=1e-12 * np.abs(a).max())
        else:
            np.testing.assert_allclose(g[k][keep], a[keep], rtol=0, atol=2e-5 * np.abs(a).max())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32c", 2e-6)])
def test_initial_tables_match_the_oracle(prec, tol):
    P = full_problem(5003, prec)
    ctx = B.from_problem(P, prec)
    T = ctx.m2m_get_sh_table(64, full=True)
    st = O.init(P, prec)
    assert_tables_close(T, st.sh, tol)
    # no symmetry: odd l and sine terms are far from zero
    F = split_table(T)[0]
    for t in (1, 3, 4, 8):                 # (1,-1), (1,1), (2,-2), (2,2)
        assert np.abs(F[t]).max() > 1e-4 * np.abs(F[0]).max(), t


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_push_in_the_expansion(prec):
    P = full_problem(4097, prec, K=128)
    ctx = B.from_problem(P, prec)
    ctx.m2m_push(40)
    g = ctx.state()
    st = O.init(P, prec)
    s = (st.x, st.y, st.z, st.vx, st.vy, st.vz)
    rmin = np.full(P.n, np.inf)
    for _ in range(40):
        s = O.kdk(*s, P.potential, P.dt, st.sh)
        rmin = np.minimum(rmin, np.sqrt(s[0].astype(np.float64) ** 2 + s[1] ** 2 + s[2] ** 2))
    assert_positions_close(g, s, resolved(rmin), prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_step_recomputes_the_expansion_on_schedule(prec):
    P = full_problem(6001, prec, K=64, period=5)
    comp = P.potential[0]
    tol = 1e-12 if prec == "fp64" else 2e-6
    ctx = B.from_problem(P, prec)
    ctx.m2m_step(20)
    g20 = ctx.state()
    T = ctx.m2m_get_sh_table(64, full=True)
    assert_tables_close(T, O.sh_tables(g20["x"], g20["y"], g20["z"], g20["w"], comp), tol)
    ctx.m2m_step(3)
    assert np.array_equal(ctx.m2m_get_sh_table(64, full=True), T)
    ctx.m2m_step(2)
    assert not np.array_equal(ctx.m2m_get_sh_table(64, full=True), T)


def test_potential_call_switches_between_the_three_expansions():
    P = full_problem(3000, "fp64", K=32, targets=False)
    ctx = B.from_problem(P, "fp64")
    ctx.m2m_push(5)
    g = ctx.state()
    tri = I.PotentialComponent("sh_tri", (40, 1e-3, 50.0, 9))
    ctx.m2m_potential([tri])
    Ft, _, _ = O.sh_tables(g["x"], g["y"], g["z"], g["w"], tri)
    assert np.abs(ctx.m2m_get_sh_table(40, triaxial=True)[:, :15].T - Ft).max() <= 1e-12 * np.abs(Ft[0]).max()
    full = I.PotentialComponent("sh_full", (48, 1e-3, 50.0, 9))
    ctx.m2m_potential([full])
    assert_tables_close(ctx.m2m_get_sh_table(48, full=True),
                        O.sh_tables(g["x"], g["y"], g["z"], g["w"], full), 1e-12)


def test_kept_forces_equal_evaluated_forces():
    P = full_problem(6001, "fp32c", K=64, period=5)
    out = []
    for keep in (True, False):
        ctx = B.from_problem(P, "fp32c")
        ctx.m2m_set_force_cache(keep)
        ctx.m2m_step(12)
        ctx.m2m_push(3)
        ctx.m2m_step(9)
        out.append((ctx.state(), ctx.m2m_get_obs()[0]))
        ctx.m2m_free()
    (g1, y1), (g0, y0) = out
    for k in ("x", "y", "z", "vx", "vy", "vz", "w"):
        assert np.array_equal(g1[k], g0[k]), k
    assert np.array_equal(y1, y0)


@pytest.mark.parametrize("prec,wtol,ytol,nsteps", [("fp64", 1e-10, 1e-10, 100), ("fp32c", 1e-4, 1e-5, 300)])
def test_weights_and_observables_on_the_gpu_orbits(prec, wtol, ytol, nsteps):
    P = full_problem(6001, prec, K=64, period=5)
    ctx = B.from_problem(P, prec)
    st = O.init(P, prec)
    for _ in range(nsteps):
        ctx.m2m_step(1)
        g = ctx.state()
        st.x, st.y, st.z, st.vx, st.vy, st.vz = (g[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz"))
        O.step(st, P, push=False)
    g = ctx.state()
    y, _, _ = ctx.m2m_get_obs()
    np.testing.assert_allclose(g["w"], st.w, rtol=wtol)
    scale = np.maximum(np.maximum(np.abs(st.y_obs), P.sigma / 0.02), 1e-300)
    err = np.abs(y - st.y_obs) / scale
    assert err.max() <= ytol, (err.max(), err.argmax())
    ctx.m2m_free()


def test_full_size_tables_and_push_sampled():
    """The workload at its full size (N = 4,000,000, K = 128, recompute
    every 50 steps) through one recompute inside m2m_step: the table
    against the oracle's expansion of the same state, then one push of a
    sample of particles."""
    P = I.make_problem("sh-full", precision="fp32c", with_target=False)
    P = P.with_targets(np.ones(P.nobs))
    comp = P.potential[0]
    ctx = B.from_problem(P, "fp32c")
    ctx.m2m_step(50)
    g = ctx.state()
    ref = O.sh_tables(g["x"], g["y"], g["z"], g["w"], comp)
    assert_tables_close(ctx.m2m_get_sh_table(128, full=True), ref, 2e-6)
    idx = np.random.default_rng(0).choice(P.n, 8192, replace=False)
    s0 = tuple(g[k][idx] for k in ("x", "y", "z", "vx", "vy", "vz"))
    ctx.m2m_push(1)
    g1 = ctx.state()
    s1 = O.kdk(*s0, P.potential, P.dt, ref)
    for a, k in zip(s1, ("x", "y", "z", "vx", "vy", "vz")):
        np.testing.assert_allclose(g1[k][idx], a, rtol=0, atol=2e-6 * np.abs(a).max())
