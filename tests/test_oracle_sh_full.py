"""Pins of the general (all l, m) multipole expansion of the oracle."""
import math

import numpy as np
import pytest

from oracle import sh as SH
from oracle import sh_full as F
from paper_1207_6403_gb300 import inputs as I


def test_real_harmonics_are_orthonormal_by_quadrature():
    """Gauss-Legendre in mu (9 points) times 17 equally spaced phi integrate
    every product of two harmonics with l <= 8 exactly."""
    L = 8
    mu, wm = np.polynomial.legendre.leggauss(L + 1)
    nphi = 2 * L + 1
    phi = 2 * math.pi * np.arange(nphi) / nphi
    M, PH = np.meshgrid(mu, phi, indexing="ij")
    s = np.sqrt(1 - M * M)
    Y = F.real_harmonics(L, (s * np.cos(PH)).ravel(), (s * np.sin(PH)).ravel(), M.ravel())
    wq = (np.outer(wm, np.full(nphi, 2 * math.pi / nphi))).ravel()
    G = (Y * wq) @ Y.T
    np.testing.assert_allclose(G, np.eye(Y.shape[0]), atol=1e-12)


def test_addition_theorem():
    """sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a.b) with P_l by Bonnet's
    recurrence."""
    g = np.random.default_rng(3)
    a, b = g.normal(size=(2, 3, 50))
    Ya = F.real_harmonics(8, *a)
    Yb = F.real_harmonics(8, *b)
    cosg = (a * b).sum(0) / np.sqrt((a * a).sum(0) * (b * b).sum(0))
    P = SH.legendre(cosg, 8)
    idx = F.index(8)
    for l in range(9):
        rows = [k for k, (ll, _) in enumerate(idx) if ll == l]
        np.testing.assert_allclose((Ya[rows] * Yb[rows]).sum(0), (2 * l + 1) / (4 * math.pi) * P[l],
                                   rtol=1e-11, atol=1e-13)


def test_truncated_series_converges_to_the_newtonian_potential():
    """|Phi_lmax - Phi| <= sum_i w_i q_i^(lmax+1) / (r_> (1 - q_i)), q = r_</r_>."""
    g = np.random.default_rng(5)
    x, y, z = g.normal(size=(3, 40)) * 0.4
    w = g.uniform(0.5, 1.5, 40)
    p = np.array([[1.7, -0.9, 1.2], [0.05, 0.1, -0.08]]).T
    for j in range(p.shape[1]):
        d = np.sqrt((p[0, j] - x) ** 2 + (p[1, j] - y) ** 2 + (p[2, j] - z) ** 2)
        exact = -np.sum(w / d)
        rp, ri = np.linalg.norm(p[:, j]), np.sqrt(x * x + y * y + z * z)
        q = np.minimum(rp, ri) / np.maximum(rp, ri)
        prev = None
        for L in (4, 8, 12):
            err = abs(F.potential(*p[:, j:j + 1], x, y, z, w, L)[0] - exact)
            bound = np.sum(w * q ** (L + 1) / (np.maximum(rp, ri) * (1 - q)))
            assert err <= bound + 1e-12
            if prev is not None and bound < 1e-3:
                assert err < prev
            prev = err


def test_axisymmetric_even_part_is_the_step_expansion_at_a_node():
    """Restricted to m = 0 and even l <= 8, the general expansion at a node
    radius equals -sum_l P_l(mu) F_l(k) of the step's expansion tables."""
    g = np.random.default_rng(7)
    n = 300
    x, y, z = g.normal(size=(3, n))
    w = g.uniform(0.5, 1.5, n) / n
    rn = SH.nodes(0.05, 20.0, 16)
    A, B = SH.coefficients(x, y, z, w, rn)
    Ft, Dt = SH.tables(A, B, rn)
    k = 9
    mu = np.array([-0.8, 0.1, 0.6])
    ph = np.array([0.3, 2.0, -1.1])
    s = np.sqrt(1 - mu * mu)
    px, py, pz = rn[k] * s * np.cos(ph), rn[k] * s * np.sin(ph), rn[k] * mu
    Yp = F.real_harmonics(8, px, py, pz)
    Yi = F.real_harmonics(8, x, y, z)
    ri = np.sqrt(x * x + y * y + z * z)
    ref = -(SH.legendre(mu, 8)[list(SH.LS)] * Ft[:, k:k + 1]).sum(0)
    out = np.zeros(3)
    for j in range(3):
        inside = ri * ri < rn[k] ** 2
        rl = np.where(inside, ri, rn[k])
        rg = np.where(inside, rn[k], ri)
        for kk, (l, m) in enumerate(F.index(8)):
            if m == 0 and l % 2 == 0:
                out[j] -= np.sum(w * 4 * math.pi / (2 * l + 1) * Yp[kk, j] * Yi[kk] * rl ** l / rg ** (l + 1))
    np.testing.assert_allclose(out, ref, rtol=1e-10)


def test_mirror_symmetric_sets_keep_even_l_and_even_nonnegative_m():
    """Particles mirrored in the three coordinate planes (a triaxial,
    reflection-symmetric model): sum w r^l Y_lm vanishes unless l and m are
    even and m >= 0."""
    g = np.random.default_rng(9)
    x, y, z = np.abs(g.normal(size=(3, 100)))
    sx, sy, sz = np.meshgrid([1, -1], [1, -1], [1, -1], indexing="ij")
    X = np.concatenate([a * x for a in sx.ravel()])
    Y = np.concatenate([a * y for a in sy.ravel()])
    Z = np.concatenate([a * z for a in sz.ravel()])
    r = np.sqrt(X * X + Y * Y + Z * Z)
    H = F.real_harmonics(8, X, Y, Z)
    for k, (l, m) in enumerate(F.index(8)):
        c = np.sum(r ** l * H[k])
        if l % 2 or m % 2 or m < 0:
            assert abs(c) < 1e-9 * np.sum(r ** l), (l, m, c)


def _cloud(n=400, seed=11):
    g = np.random.default_rng(seed)
    x, y, z = g.normal(size=(3, n)) * np.array([[1.0], [0.7], [0.4]])     # triaxial
    return x, y, z, g.uniform(0.5, 1.5, n) / n


def test_tabulated_expansion_is_exact_at_the_nodes():
    """At a node radius the tabulated potential is the direct double sum of
    the same truncation (no interpolation there)."""
    x, y, z, w = _cloud()
    rn = SH.nodes(0.02, 30.0, 24)
    A, B = F.coefficients_nodes(x, y, z, w, rn, 6)
    Ft, Dt = F.tables_nodes(A, B, rn, 6)
    g = np.random.default_rng(2)
    for k in (3, 11, 17):
        d = g.normal(size=(3, 4))
        d = d / np.linalg.norm(d, axis=0) * rn[k]
        np.testing.assert_allclose(F.potential_nodes(*d, Ft, Dt, rn, 6),
                                   F.potential(*d, x, y, z, w, 6), rtol=1e-11)


def test_tabulated_axisymmetric_part_is_the_step_expansion_everywhere():
    """Keeping only m = 0 and even l, the tabulated general expansion equals
    the step's axisymmetric expansion at any point (interpolated between
    nodes and by the laws outside them alike)."""
    x, y, z, w = _cloud()
    rn = SH.nodes(0.05, 20.0, 16)
    A, B = F.coefficients_nodes(x, y, z, w, rn, 8)
    Ft, Dt = F.tables_nodes(A, B, rn, 8)
    keep = np.array([m == 0 and l % 2 == 0 for l, m in F.index(8)])
    Ft[~keep] = 0.0
    Dt[~keep] = 0.0
    Fa, Da = SH.tables(*SH.coefficients(x, y, z, w, rn), rn)
    g = np.random.default_rng(4)
    p = g.normal(size=(3, 30)) * np.geomspace(0.01, 40.0, 30)
    np.testing.assert_allclose(F.potential_nodes(*p, Ft, Dt, rn, 8), SH.potential(*p, Fa, Da, rn),
                               rtol=1e-11, atol=1e-13)


def test_tabulated_monopole_obeys_gauss_at_the_last_node():
    x, y, z, w = _cloud()
    rn = SH.nodes(0.05, 20.0, 16)
    A, B = F.coefficients_nodes(x, y, z, w, rn, 2)
    Ft, _ = F.tables_nodes(A, B, rn, 2)
    inside = (x * x + y * y) + z * z < rn[-1] ** 2
    Y00 = 1.0 / math.sqrt(4 * math.pi)
    assert Ft[0, -1] * Y00 == pytest.approx(np.sum(w[inside]) / rn[-1], rel=1e-13)


def test_tabulated_force_axisymmetric_part_is_the_step_force():
    """m = 0, even l only: the general force equals the step expansion's
    force at any point, on and off the z axis."""
    x, y, z, w = _cloud()
    rn = SH.nodes(0.05, 20.0, 16)
    A, B = F.coefficients_nodes(x, y, z, w, rn, 8)
    Ft, Dt = F.tables_nodes(A, B, rn, 8)
    keep = np.array([m == 0 and l % 2 == 0 for l, m in F.index(8)])
    Ft[~keep] = 0.0
    Dt[~keep] = 0.0
    Fa, Da = SH.tables(*SH.coefficients(x, y, z, w, rn), rn)
    g = np.random.default_rng(6)
    p = g.normal(size=(3, 30)) * np.geomspace(0.01, 40.0, 30)
    p[:2, :3] = 0.0                                        # on the z axis
    ref = np.stack(SH.acceleration(*p, Fa, Da, rn))
    np.testing.assert_allclose(F.acceleration_nodes(*p, Ft, Dt, rn, 8), ref, rtol=1e-10,
                               atol=1e-12 * np.abs(ref).max())


def test_tabulated_force_tangential_part_is_minus_the_angular_gradient():
    """On a sphere r = const the tabulated potential is a finite sum of
    harmonics: its derivative along a tangent t (central difference on the
    sphere, error O(h^2)) is -a.t for every l, m (triaxial cloud, l <= 6),
    on and near the z axis too."""
    x, y, z, w = _cloud()
    rn = SH.nodes(0.02, 30.0, 24)
    A, B = F.coefficients_nodes(x, y, z, w, rn, 6)
    Ft, Dt = F.tables_nodes(A, B, rn, 6)
    g = np.random.default_rng(8)
    pts = g.normal(size=(3, 12))
    pts[:, 0] = [0.0, 0.0, 1.0]
    pts[:, 1] = [1e-3, 0.0, 1.0]
    pts = pts / np.linalg.norm(pts, axis=0) * 1.3
    a = F.acceleration_nodes(*pts, Ft, Dt, rn, 6)
    h = 1e-5
    for j in range(pts.shape[1]):
        p = pts[:, j]
        nrm = p / np.linalg.norm(p)
        for v in (np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0])):
            t = v - nrm * (v @ nrm)
            if np.linalg.norm(t) < 0.3:
                continue
            t = t / np.linalg.norm(t)
            # move on the sphere: rotate p towards t by the angle h
            pp = np.linalg.norm(p) * (np.cos(h) * nrm + np.sin(h) * t)
            pm = np.linalg.norm(p) * (np.cos(h) * nrm - np.sin(h) * t)
            dphi = (F.potential_nodes(*pp[:, None], Ft, Dt, rn, 6)[0]
                    - F.potential_nodes(*pm[:, None], Ft, Dt, rn, 6)[0]) / (2 * h * np.linalg.norm(p))
            assert -a[:, j] @ t == pytest.approx(dphi, rel=1e-6, abs=1e-9 * np.abs(a).max())


def _mirrored(n=300, seed=13):
    g = np.random.default_rng(seed)
    x, y, z = np.abs(g.normal(size=(3, n))) * np.array([[1.0], [0.8], [0.6]])
    sx, sy, sz = np.meshgrid([1, -1], [1, -1], [1, -1], indexing="ij")
    X = np.concatenate([a * x for a in sx.ravel()])
    Y = np.concatenate([a * y for a in sy.ravel()])
    Z = np.concatenate([a * z for a in sz.ravel()])
    w = np.tile(g.uniform(0.5, 1.5, n) / n, 8)
    return X, Y, Z, w


def test_triaxial_expansion_is_the_full_expansion_of_a_triaxial_set():
    """For particles mirrored in the three coordinate planes the 15 terms of
    the triaxial expansion (even l, even m >= 0, l <= 8) carry the whole
    lmax = 8 expansion: their node tables are the full tables' rows, every
    other row vanishes, and the tabulated potential and force of the subset
    are those of all 81 terms (at nodes, between them and outside them)."""
    from oracle import sh as SH0
    X, Y, Z, w = _mirrored()
    rn = SH0.nodes(0.05, 5.0, 48)
    Af, Bf = F.coefficients_nodes(X, Y, Z, w, rn, 8)
    Ff, Df = F.tables_nodes(Af, Bf, rn, 8)
    Ft, Dt, _ = F.tri_tables(X, Y, Z, w, rn)
    terms = F.triaxial_terms(8)
    assert len(terms) == 15
    idx = F.index(8)
    scale = np.abs(Ff).max()
    for k, t in enumerate(idx):
        if t in terms:
            j = terms.index(t)
            assert np.abs(Ft[j] - Ff[k]).max() <= 1e-12 * scale and np.abs(Dt[j] - Df[k]).max() <= 1e-10 * scale
        else:
            assert np.abs(Ff[k]).max() <= 1e-12 * scale, t
    g = np.random.default_rng(3)
    p = g.normal(size=(3, 200)) * np.array([[2.0], [1.5], [1.0]])
    p[:, :10] *= 5.0                       # beyond the last node
    p[:, 10:20] *= 0.005                   # inside the first
    phi_f = F.potential_nodes(*p, Ff, Df, rn, 8)
    phi_t = F.tri_potential(*p, Ft, Dt, rn)
    np.testing.assert_allclose(phi_t, phi_f, rtol=1e-11, atol=1e-12 * np.abs(phi_f).max())
    a_f = F.acceleration_nodes(*p, Ff, Df, rn, 8)
    a_t = F.tri_acceleration(*p, Ft, Dt, rn)
    np.testing.assert_allclose(a_t, a_f, rtol=1e-10, atol=1e-11 * np.abs(a_f).max())


def test_full_expansion_of_the_step_on_a_set_with_no_symmetry():
    """The step's full expansion (kind 'sh_full': every l <= 4, every m) of
    a rotated and shifted triaxial set: every harmonic is present (odd l
    and sine terms included), and at node radii its potential is the
    direct double sum of the same truncation over the particles inside
    r_max."""
    from oracle import m2m as M
    P = I.make_problem("sh-full", n=3000, precision="fp64", with_target=False)
    x, y, z = P.pos
    w = P.w0
    comp = P.potential[0]
    Ft, Dt, rn = M.sh_tables(x, y, z, w, comp)
    assert Ft.shape == (25, 128)
    mono = np.abs(Ft[0]).max()
    for t in range(1, 25):                 # (1,-1), (1,0), .., (4,4): none vanishes
        assert np.abs(Ft[t]).max() > 1e-6 * mono, t
    inside = np.sqrt(x * x + y * y + z * z) < rn[-1]
    g = np.random.default_rng(5)
    for k in (20, 64, 100):
        d = g.normal(size=(3, 4))
        d = d / np.linalg.norm(d, axis=0) * rn[k]
        np.testing.assert_allclose(M.potential(*d, P.potential, (Ft, Dt, rn)),
                                   F.potential(*d, x[inside], y[inside], z[inside], w[inside], 4), rtol=1e-11)
