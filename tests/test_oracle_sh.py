"""Pins of the spherical-harmonic potential of the oracle: explicit Legendre
polynomials, the exact multipole series of a ring of mass (at the nodes,
beyond the outermost node and inside the innermost one), the analytic
Hernquist monopole, vanishing l >= 2 terms of a spherical sample, Gauss's law
for the enclosed mass, and the acceleration against finite differences of the
exact ring series."""
import math

import numpy as np
import pytest

from oracle import sh as SH
from paper_1207_6403_gb300 import inputs as I


def test_legendre_against_explicit_polynomials():
    mu = np.linspace(-1, 1, 41)
    P = SH.legendre(mu)
    np.testing.assert_allclose(P[2], (3 * mu ** 2 - 1) / 2, atol=1e-15)
    np.testing.assert_allclose(P[4], (35 * mu ** 4 - 30 * mu ** 2 + 3) / 8, atol=1e-14)
    np.testing.assert_allclose(P[6], (231 * mu ** 6 - 315 * mu ** 4 + 105 * mu ** 2 - 5) / 16, atol=1e-13)
    np.testing.assert_allclose(P[8], (6435 * mu ** 8 - 12012 * mu ** 6 + 6930 * mu ** 4 - 1260 * mu ** 2 + 35) / 128,
                               atol=1e-13)
    h = 1e-6
    dP = SH.legendre_deriv(mu[1:-1])
    fd = (SH.legendre(mu[1:-1] + h) - SH.legendre(mu[1:-1] - h)) / (2 * h)
    np.testing.assert_allclose(dP, fd, atol=1e-7)


def _ring(n=4096, a=1.3, z0=0.0, M=1.0):
    phi = 2 * math.pi * (np.arange(n) + 0.5) / n
    return a * np.cos(phi), a * np.sin(phi), np.full(n, z0), np.full(n, M / n)


def _ring_series(r, mu, a=1.3, M=1.0):
    """Exact m=0, even-l <= 8 multipole series of a ring in z = 0."""
    P = SH.legendre(mu)
    P0 = SH.legendre(np.array(0.0))
    tot = 0.0
    for l in SH.LS:
        rl, rg = np.minimum(r, a), np.maximum(r, a)
        tot = tot - M * P0[l] * P[l] * rl ** l / rg ** (l + 1)
    return tot


def test_ring_node_values_equal_the_exact_series():
    x, y, z, w = _ring()
    rn = SH.nodes(0.01, 50.0, 64)
    A, B = SH.coefficients(x, y, z, w, rn)
    F, D = SH.tables(A, B, rn)
    for mu in (0.0, 0.3, -0.7, 1.0):
        phi = -np.sum(SH.legendre(np.full(rn.shape, mu))[list(SH.LS)] * F, axis=0)
        np.testing.assert_allclose(phi, _ring_series(rn, mu), rtol=1e-12, atol=1e-14)


def test_acceleration_at_nodes_matches_gradient_of_exact_series():
    x, y, z, w = _ring()
    rn = SH.nodes(0.01, 50.0, 64)
    F, D = SH.tables(*SH.coefficients(x, y, z, w, rn), rn)
    k = np.array([10, 30, 40, 55])
    th = np.array([0.4, 1.1, 2.0, 2.7])
    ph = np.array([0.3, 1.9, 4.0, 5.5])
    r = rn[k]
    px, py, pz = r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)
    ax, ay, az = SH.acceleration(px, py, pz, F, D, rn)

    def phi(X, Y, Z):
        R = np.sqrt(X * X + Y * Y + Z * Z)
        return _ring_series(R, Z / R)
    h = 1e-6
    gx = (phi(px + h, py, pz) - phi(px - h, py, pz)) / (2 * h)
    gy = (phi(px, py + h, pz) - phi(px, py - h, pz)) / (2 * h)
    gz = (phi(px, py, pz + h) - phi(px, py, pz - h)) / (2 * h)
    for a, g in ((ax, gx), (ay, gy), (az, gz)):
        np.testing.assert_allclose(a, -g, rtol=1e-5, atol=1e-7)


def test_hernquist_monopole_and_vanishing_higher_multipoles():
    pos, vel = I.hernquist_isotropic(200_000, 21)
    w = np.full(pos.shape[1], 1.0 / pos.shape[1])
    rmax = 100.0
    rn = SH.nodes(0.01, rmax, 128)
    A, B = SH.coefficients(*pos, w, rn)
    F, D = SH.tables(A, B, rn)
    # monopole: the sample is a Hernquist sphere truncated at rmax and scaled
    # to unit mass, whose potential is -(1/(1+r) - 1/(1+rmax)^2) / M(<rmax)
    Mtot = (rmax / (1 + rmax)) ** 2
    exact = (1.0 / (1 + rn) - 1.0 / (1 + rmax) ** 2) / Mtot
    outer = (rn > 0.3) & (rn < 20)
    np.testing.assert_allclose(F[0][outer], exact[outer], rtol=0.005)
    # inside, sum w/r_i over few central particles is heavy-tailed: looser
    inner = (rn > 0.05) & (rn <= 0.3)
    np.testing.assert_allclose(F[0][inner], exact[inner], rtol=0.03)
    # l >= 2 of an isotropic sample: zero within shot noise.  With mu uniform,
    # E[P_l] = 0 and E[P_l^2] = 1/(2l+1), so A_l(r_k) and B_l(r_k) (sums over
    # disjoint particles) have variances sum w^2 r^(2l)/(2l+1) and
    # sum w^2 r^-(2l+2)/(2l+1)
    r = np.sort(np.sqrt((pos ** 2).sum(0)))
    ws = w[0]
    below = np.searchsorted(r, rn)
    inside = r < rmax
    sel = (rn > 0.02) & (rn < 50)
    for n, l in enumerate(SH.LS[1:], start=1):
        ca = np.concatenate([[0.0], np.cumsum(ws ** 2 * r ** (2 * l))])
        cb = np.concatenate([[0.0], np.cumsum(np.where(inside, ws ** 2 * r ** (-2.0 * l - 2), 0.0))])
        va = ca[below] / (2 * l + 1)
        vb = (cb[-1] - cb[below]) / (2 * l + 1)
        sd = np.sqrt(va / rn ** (2 * l + 2) + vb * rn ** (2 * l))
        # the terms are far from Gaussian (P_8 peaks at the poles, r^-(2l+2)
        # weights the innermost particles of B), so the tail is wide; the
        # median (0.67 for a normal variate) shows the scale is right
        q = np.abs(F[n][sel]) / sd[sel]
        assert q.max() < 8 and np.median(q) < 1.5, l


def _fd_accel(px, py, pz, phi, h=1e-6):
    gx = (phi(px + h, py, pz) - phi(px - h, py, pz)) / (2 * h)
    gy = (phi(px, py + h, pz) - phi(px, py - h, pz)) / (2 * h)
    gz = (phi(px, py, pz + h) - phi(px, py, pz - h)) / (2 * h)
    return -gx, -gy, -gz


def _ring_phi(X, Y, Z):
    R = np.sqrt(X * X + Y * Y + Z * Z)
    return _ring_series(R, Z / R)


def test_exterior_law_beyond_the_last_node_is_the_exact_series():
    x, y, z, w = _ring()
    rn = SH.nodes(0.1, 5.0, 32)
    F, D = SH.tables(*SH.coefficients(x, y, z, w, rn), rn)
    r = np.array([5.0, 7.0, 12.0, 40.0])
    th = np.array([0.3, 1.2, 1.9, 2.9])
    px, py, pz = r * np.sin(th) * np.cos(0.7), r * np.sin(th) * np.sin(0.7), r * np.cos(th)
    np.testing.assert_allclose(SH.potential(px, py, pz, F, D, rn), _ring_phi(px, py, pz), rtol=1e-12)
    for a, g in zip(SH.acceleration(px, py, pz, F, D, rn), _fd_accel(px, py, pz, _ring_phi)):
        np.testing.assert_allclose(a, g, rtol=1e-5, atol=1e-9)


def test_uniform_core_inside_the_first_node():
    # no mass inside r_0: the exact l = 0 force is 0 and the l = 2 force is
    # linear in r, which is what the core law gives; l >= 4 terms are O(r^3)
    x, y, z, w = _ring()
    rn = SH.nodes(0.1, 5.0, 32)
    F, D = SH.tables(*SH.coefficients(x, y, z, w, rn), rn)
    r = np.array([0.02, 0.05, 0.09])
    th = np.array([0.5, 1.0, 2.5])
    px, py, pz = r * np.sin(th), np.zeros(3), r * np.cos(th)
    got = SH.acceleration(px, py, pz, F, D, rn)
    exp = _fd_accel(px, py, pz, _ring_phi, h=1e-7)
    scale = np.abs(np.array(exp)).max()
    for a, g in zip(got, exp):
        np.testing.assert_allclose(a, g, atol=2e-3 * scale)
    assert SH.acceleration(np.zeros(1), np.zeros(1), np.zeros(1), F, D, rn)[0][0] == 0.0


def test_gauss_law_at_the_last_node():
    # at r_(K-1) = rmax nothing lies further out, so F_0 r = enclosed mass and
    # the radial force is -M/r^2
    pos, _ = I.hernquist_isotropic(50_000, 5)
    w = np.random.default_rng(3).uniform(0.5, 1.5, pos.shape[1]) / pos.shape[1]
    rn = SH.nodes(0.01, 30.0, 64)
    F, D = SH.tables(*SH.coefficients(*pos, w, rn), rn)
    r = np.sqrt((pos ** 2).sum(0))
    M = w[(pos[0] * pos[0] + pos[1] * pos[1]) + pos[2] * pos[2] < 30.0 ** 2].sum()
    assert F[0, -1] * 30.0 == pytest.approx(M, rel=1e-13)
    assert D[0, -1] == pytest.approx(-M / 900.0, rel=1e-13)
    assert (r >= 30.0).any()


def test_node_side_uses_r2_in_the_state_precision():
    # a float32 position whose float32 r^2 equals the float64 node square
    # exactly is on the upper side (half-open), whatever its float64 r^2
    rn = np.array([0.5, 1.0, 2.0])
    x = np.array([1.0, np.nextafter(np.float32(1.0), np.float32(0))], dtype=np.float32)
    j = SH.node_side(x, np.zeros(2, np.float32), np.zeros(2, np.float32), rn)
    assert list(j) == [2, 1]
    j64 = SH.node_side(np.array([2.0, 1.999999]), np.zeros(2), np.zeros(2), rn)
    assert list(j64) == [3, 2]


def _sh_problem(n=3000, period=5, K=128):
    P = I.make_problem("sh-selfcons", n=n, with_target=False)
    P.potential = [I.PotentialComponent("sh", (K, 1e-3, 100.0, period))]
    return P.with_targets(np.ones(P.nobs))


def test_step_recomputes_the_expansion_every_period_from_the_new_state():
    from oracle import m2m as O
    P = _sh_problem(period=4)
    st = O.init(P)
    np.testing.assert_array_equal(st.sh[0], O.sh_tables(st.x, st.y, st.z, st.w, P.potential[0])[0])
    seen = [st.sh[0]]
    for t in range(1, 10):
        O.step(st, P)
        if t % 4 == 0:
            assert not np.array_equal(st.sh[0], seen[-1]), t
            np.testing.assert_array_equal(st.sh[0], O.sh_tables(st.x, st.y, st.z, st.w, P.potential[0])[0])
        else:
            assert st.sh[0] is seen[-1], t
        seen.append(st.sh[0])


def test_leapfrog_in_a_frozen_expansion_conserves_energy():
    # the force is minus the gradient of the same expansion up to the
    # interpolation between nodes, so the energy error of a KDK orbit in a
    # frozen expansion of a flattened disc + bulge falls as the nodes get
    # denser; a wrong sign or a dropped term of the force would not
    from oracle import m2m as O
    pos, vel = I.disc_bulge_realisation(4000, 11)
    w = np.full(pos.shape[1], 1.0 / pos.shape[1])
    med = {}
    for K in (128, 1024):
        comp = I.PotentialComponent("sh", (K, 1e-3, 100.0, 10 ** 9))
        sh = O.sh_tables(*pos, w, comp)
        x, y, z = pos
        vx, vy, vz = vel
        E0 = 0.5 * (vx * vx + vy * vy + vz * vz) + SH.potential(x, y, z, *sh)
        for _ in range(300):
            x, y, z, vx, vy, vz = O.kdk(x, y, z, vx, vy, vz, [comp], 0.01, sh)
        E1 = 0.5 * (vx * vx + vy * vy + vz * vz) + SH.potential(x, y, z, *sh)
        med[K] = np.median(np.abs(E1 / E0 - 1))
    assert med[1024] < 1.5e-4
    assert med[128] > 5 * med[1024]
