"""GPU parity of the triaxial expansion (potential kind 'sh_tri': even
l <= 8, even m >= 0) and of the (E, L^2) prior cells: node tables against
the oracle's direct node sums, pushes, the recompute schedule inside
m2m_step, the edge cases of the radial laws and of the angular terms, the
weights and observables on the GPU's own orbits, and the full-size
triaxial workload on samples.

Tolerances, as for the axisymmetric expansion:
* FP64: double side sums in another order than the oracle's, so the tables
  agree to 1e-12 of the monopole scale (every term, the small high-(l, m)
  ones included, is held to that absolute bound); positions after a push
  to 1e-10 relative.
* FP32C: float per-particle terms (the weights enter truncated to float),
  exact fixed-point sums: tables to 2e-6 of the monopole scale; the force
  is evaluated in float, so positions agree to 2e-5 of their range after a
  few tens of steps.
The model has a density cusp (Hernquist-like): orbits through the centre
are not resolved by dt and amplify rounding differences, so trajectories
are compared for the particles whose oracle orbit stays outside r = 0.05,
and long runs are checked on the GPU's own orbits.

Prior cells: with an analytic potential the energies are the same
sequence of operations in the state precision on both sides and every
(E, L^2) cell matches.  With the triaxial expansion the GPU's potential is
its own float (or double) evaluation of the tables and the oracle's is
float64 rounded to the state precision, so a particle whose E or L^2 lies
within rounding of a cell edge may fall on either side: every other
particle's cell must match, and those at an edge differ by one E or L^2
cell at most.
"""
import numpy as np
import pytest

from oracle import m2m as O
from oracle import sh as SH
from paper_1207_6403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402

_CACHE = {}
NT = 15


def tri_problem(n, prec, K=64, period=5, seed=12, targets=True, prior=None):
    key = (n, prec, K, period, seed, targets, repr(prior))
    if key not in _CACHE:
        P = I.make_problem("sh-tri", n=n, precision=prec, seed_model=seed, seed_target=seed + 1,
                           with_target=targets)
        P.potential = [I.PotentialComponent("sh_tri", (K, 1e-3, 100.0, period))]
        P.prior = prior or I.PriorSpec("flat")
        if targets:
            Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
            P = P.with_targets(Y)
        else:
            P = P.with_targets(np.ones(P.nobs))
        _CACHE[key] = P
    return _CACHE[key]


def split_table(T):
    return T[:, 0:15].T, T[:, 15:30].T, T[:, 30:45].T, T[:, 45:60].T, T[:, 60]


def assert_tables_close(T, ref, tol):
    F, SF, D, SD, rk = split_table(T)
    Fo, Do, rn = ref
    assert Fo.shape == (NT, len(rn))
    np.testing.assert_array_equal(rk, rn if tol < 1e-9 else rn.astype(np.float32))
    sF, sD = np.abs(Fo[0]).max(), np.abs(Do[0]).max()
    assert np.abs(F - Fo).max() <= tol * sF, (np.abs(F - Fo).max() / sF, np.unravel_index(np.abs(F - Fo).argmax(), F.shape))
    assert np.abs(D - Do).max() <= tol * sD, (np.abs(D - Do).max() / sD, np.unravel_index(np.abs(D - Do).argmax(), D.shape))
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
    P = tri_problem(5003, prec)
    ctx = B.from_problem(P, prec)
    T = ctx.m2m_get_sh_table(64, triaxial=True)
    st = O.init(P, prec)
    assert_tables_close(T, st.sh, tol)
    # the model is triaxial: the m = 2 terms are far from zero
    F = split_table(T)[0]
    assert np.abs(F[2]).max() > 1e-3 * np.abs(F[0]).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_push_in_the_expansion(prec):
    P = tri_problem(4097, prec, K=128)
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
    P = tri_problem(6001, prec, K=64, period=5)
    comp = P.potential[0]
    tol = 1e-12 if prec == "fp64" else 2e-6
    ctx = B.from_problem(P, prec)
    ctx.m2m_step(20)
    g20 = ctx.state()
    T = ctx.m2m_get_sh_table(64, triaxial=True)
    assert_tables_close(T, O.sh_tables(g20["x"], g20["y"], g20["z"], g20["w"], comp), tol)
    ctx.m2m_step(3)
    g = ctx.state()
    assert np.array_equal(ctx.m2m_get_sh_table(64, triaxial=True), T)
    st = O.init(P, prec)
    rmin = np.full(P.n, np.inf)
    for _ in range(23):
        O.step(st, P)
        rmin = np.minimum(rmin, np.sqrt(st.x.astype(np.float64) ** 2 + st.y ** 2 + st.z ** 2))
    assert_positions_close(g, (st.x, st.y, st.z, st.vx, st.vy, st.vz), resolved(rmin), prec)
    ctx.m2m_step(2)
    assert not np.array_equal(ctx.m2m_get_sh_table(64, triaxial=True), T)


def test_edge_cases_origin_axes_outside_inside_and_on_a_node():
    P = tri_problem(2000, "fp64", K=32, targets=False)
    rn = SH.nodes(1e-3, 100.0, 32)
    x, y, z = (a.copy() for a in P.pos)
    # r = 0; beyond rmax (left out of the sums, exterior law); inside r_0
    # (interior law); exactly on nodes 0, 5 and K-1 (upper side); on the
    # z axis (mu = +-1, u = 0) and on the x and y axes (mu = 0)
    pts = [(0.0, 0.0, 0.0), (150.0, 20.0, -40.0), (2e-4, -3e-4, 1e-4), (rn[0], 0.0, 0.0), (0.0, 0.0, -rn[5]),
           (0.0, rn[31], 0.0), (0.0, 0.0, 1.5), (0.0, 0.0, -0.7), (2.5, 0.0, 0.0), (0.0, -0.3, 0.0)]
    for k, (a, b, c) in enumerate(pts):
        x[k], y[k], z[k] = a, b, c
    P2 = I.Problem(**{**P.__dict__, "pos": np.stack([x, y, z])})
    P2 = P2.with_targets(np.ones(P2.nobs))
    ctx = B.from_problem(P2, "fp64")
    st = O.init(P2, "fp64")
    assert_tables_close(ctx.m2m_get_sh_table(32, triaxial=True), st.sh, 1e-12)
    ctx.m2m_push(3)
    g = ctx.state()
    s = (st.x, st.y, st.z, st.vx, st.vy, st.vz)
    for _ in range(3):
        s = O.kdk(*s, P2.potential, P2.dt, st.sh)
    m = len(pts)
    for a, k in zip(s, ("x", "y", "z", "vx", "vy", "vz")):
        np.testing.assert_allclose(g[k][:m], a[:m], rtol=1e-12, atol=1e-15)


def test_potential_call_switches_expansions_and_rejects_a_bad_descriptor():
    P = tri_problem(3000, "fp64", K=32, targets=False)
    ctx = B.from_problem(P, "fp64")
    ctx.m2m_push(7)
    g = ctx.state()
    # to the axisymmetric expansion and back, with new node counts
    sh = I.PotentialComponent("sh", (40, 1e-3, 50.0, 9))
    ctx.m2m_potential([sh])
    F, D, rn = O.sh_tables(g["x"], g["y"], g["z"], g["w"], sh)
    T = ctx.m2m_get_sh_table(40)
    assert np.abs(T[:, 0:5].T - F).max() <= 1e-12 * np.abs(F[0]).max()
    tri = I.PotentialComponent("sh_tri", (48, 1e-3, 50.0, 9))
    ctx.m2m_potential([tri])
    assert_tables_close(ctx.m2m_get_sh_table(48, triaxial=True), O.sh_tables(g["x"], g["y"], g["z"], g["w"], tri),
                        1e-12)
    with pytest.raises(B.M2MError) as e:
        ctx.m2m_potential([I.PotentialComponent("sh_tri", (48, 1e-3, 50.0, 0))])
    assert e.value.code == -1


@pytest.mark.parametrize("prec,wtol,ytol,nsteps", [("fp64", 1e-10, 1e-10, 100), ("fp32c", 1e-4, 1e-5, 300)])
def test_weights_and_observables_on_the_gpu_orbits(prec, wtol, ytol, nsteps):
    """Every step: the GPU steps once; the oracle takes the GPU's new
    positions and does the rest of the step (scatter with the old weights,
    residual, update, triaxial recompute every 5 steps)."""
    P = tri_problem(6001, prec, K=64, period=5)
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


# ------------------------------------------------------------ (E, L^2) cells
def _edges(lo, hi, n):
    return lo + np.arange(1, n) * ((hi - lo) / n)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_e_l2_cells_with_an_analytic_potential_bit_exact(prec):
    P = I.make_problem("moving-priors", n=30007, precision=prec)
    P.prior = I.PriorSpec("e_l2", 24, 12, 10)
    P = P.with_targets(np.ones(P.nobs))
    ctx = B.from_problem(P, prec)
    ctx.m2m_push(3)
    _, pc = ctx.m2m_get_cells(with_prior=True)
    st = O.init(P, prec)
    s = (st.x, st.y, st.z, st.vx, st.vy, st.vz)
    for _ in range(3):
        s = O.kdk(*s, P.potential, P.dt)
    ref = O.prior_cells(*s, P.prior, P.potential)
    assert np.array_equal(pc.cpu().numpy(), ref)
    assert len(np.unique(ref)) > 30           # many cells of the grid are populated


@pytest.mark.parametrize("prec,rel", [("fp64", 1e-12), ("fp32c", 1e-5)])
def test_e_l2_cells_in_the_triaxial_expansion(prec, rel):
    prior = I.PriorSpec("e_l2", 64, 32, 25)
    P = tri_problem(20011, prec, K=64, period=5, targets=False, prior=prior)
    ctx = B.from_problem(P, prec)
    ctx.m2m_push(3)
    _, pc = ctx.m2m_get_cells(with_prior=True)
    pc = pc.cpu().numpy()
    g = ctx.state()
    st = O.init(P, prec)
    s = tuple(g[k] for k in ("x", "y", "z", "vx", "vy", "vz"))
    ref = O.prior_cells(*s, P.prior, P.potential, st.sh)
    # E and L^2 of the oracle at the GPU's state; particles near an edge
    x, y, z, vx, vy, vz = (np.asarray(a, np.float64) for a in s)
    E = 0.5 * ((vx * vx + vy * vy) + vz * vz) + O.potential(*s[:3], P.potential, st.sh).astype(np.float64)
    L2 = (y * vz - z * vy) ** 2 + (z * vx - x * vz) ** 2 + (x * vy - y * vx) ** 2
    eE = _edges(E.min(), E.max(), prior.nE)
    eL = _edges(0.0, L2.max(), prior.nL)
    dE = np.min(np.abs(E[:, None] - eE[None, :]), axis=1) <= rel * (E.max() - E.min()) + rel * np.abs(E)
    dL = np.min(np.abs(L2[:, None] - eL[None, :]), axis=1) <= rel * L2.max()
    near = dE | dL
    assert near.mean() < 0.01
    far = ~near
    assert np.array_equal(pc[far], ref[far])
    iEg, iLg = np.divmod(pc[near], prior.nL)
    iEo, iLo = np.divmod(ref[near], prior.nL)
    assert np.all((np.abs(iEg - iEo) <= 1) & (np.abs(iLg - iLo) <= 1))


def test_full_size_triaxial_tables_and_push_sampled():
    """The triaxial workload at its full size (N = 4,000,000, K = 256,
    recompute every 50 steps) through one recompute inside m2m_step: the
    table against the oracle's expansion of the same state, then one push
    of a sample of particles."""
    P = I.make_problem("sh-tri", precision="fp32c", with_target=False)
    P = P.with_targets(np.ones(P.nobs))
    comp = P.potential[0]
    ctx = B.from_problem(P, "fp32c")
    ctx.m2m_step(50)
    g = ctx.state()
    ref = O.sh_tables(g["x"], g["y"], g["z"], g["w"], comp)
    T = ctx.m2m_get_sh_table(256, triaxial=True)
    assert_tables_close(T, ref, 2e-6)
    idx = np.random.default_rng(0).choice(P.n, 8192, replace=False)
    s0 = tuple(g[k][idx] for k in ("x", "y", "z", "vx", "vy", "vz"))
    ctx.m2m_push(1)
    g1 = ctx.state()
    s1 = O.kdk(*s0, P.potential, P.dt, ref)
    for a, k in zip(s1, ("x", "y", "z", "vx", "vy", "vz")):
        np.testing.assert_allclose(g1[k][idx], a, rtol=0, atol=2e-6 * np.abs(a).max())


def test_kept_forces_equal_evaluated_forces():
    """As for the axisymmetric expansion: FP32C steps with the force kept
    between pushes equal the steps that evaluate it twice, bit for bit."""
    P = tri_problem(6001, "fp32c", K=64, period=5)
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
