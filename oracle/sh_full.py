"""The general multipole expansion (every l <= lmax, every m) of the
weighted particles (oracle; test infrastructure only).  The self-consistent
potential of the step (:mod:`oracle.sh`) keeps the axisymmetric, even-l
part; this module is its non-axisymmetric generalisation, for triaxial
models, written as direct sums with no radial nodes.

Real spherical harmonics, orthonormal on the unit sphere:
  Y_l0  = N_l0 P_l^0(mu),
  Y_lm  = sqrt(2) N_lm P_l^m(mu) cos(m phi),    m > 0,
  Y_l-m = sqrt(2) N_lm P_l^m(mu) sin(m phi),    m > 0,
  N_lm  = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),  mu = cos theta,
with P_l^m the associated Legendre functions without the Condon-Shortley
phase (its sign cancels in every product Y_lm Y_lm).  The potential of
particles of weight w_i (G = 1) truncated at lmax:
  Phi(x) = - sum_i w_i sum_(l <= lmax) sum_m 4 pi/(2l+1) Y_lm(x^) Y_lm(x_i^)
                    r_<^l / r_>^(l+1),
r_< and r_> the smaller and larger of |x| and |x_i|; by the addition
theorem the inner sum over m is P_l(x^ . x_i^) and the full series is
-sum_i w_i / |x - x_i|.
"""
import math

import numpy as np


def assoc_legendre(lmax, mu):
    """P_l^m(mu) for 0 <= m <= l <= lmax (no Condon-Shortley phase), as a
    dict {(l, m): array}, by the standard recurrences in l at fixed m."""
    mu = np.asarray(mu, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    P = {}
    pmm = np.ones_like(mu)
    for m in range(lmax + 1):
        if m > 0:
            pmm = pmm * (2 * m - 1) * s               # P_m^m = (2m-1)!! s^m
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = (2 * m + 1) * mu * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * mu * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    return P


def index(lmax):
    """(l, m) of every real harmonic up to lmax, m = -l..l in order."""
    return [(l, m) for l in range(lmax + 1) for m in range(-l, l + 1)]


def triaxial_terms(lmax):
    """(l, m) of the harmonics a triaxial (mirror-symmetric about the three
    coordinate planes) set of particles can have: even l, even m >= 0 (the
    cosine harmonics); the others vanish (see the pins).  At lmax = 8: 15
    terms."""
    return [(l, m) for l in range(0, lmax + 1, 2) for m in range(0, l + 1, 2)]


def _rows(lmax, terms):
    """Rows of :func:`real_harmonics` for the given terms (all by default)."""
    idx = index(lmax)
    return list(range(len(idx))) if terms is None else [idx.index(t) for t in terms]


def real_harmonics(lmax, x, y, z):
    """Y_lm at the directions of (x, y, z), shape ((lmax+1)^2, n) in the
    order of :func:`index`; the direction of the origin is taken as +z."""
    x, y, z = (np.asarray(a, dtype=np.float64) for a in (x, y, z))
    r = np.sqrt(x * x + y * y + z * z)
    rs = np.where(r > 0, r, 1.0)
    mu = np.where(r > 0, z / rs, 1.0)
    phi = np.arctan2(y, x)
    P = assoc_legendre(lmax, mu)
    out = []
    for l, m in index(lmax):
        am = abs(m)
        N = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
        if m == 0:
            out.append(N * P[(l, 0)])
        elif m > 0:
            out.append(math.sqrt(2.0) * N * P[(l, am)] * np.cos(am * phi))
        else:
            out.append(math.sqrt(2.0) * N * P[(l, am)] * np.sin(am * phi))
    return np.stack(out)


def potential(px, py, pz, x, y, z, w, lmax):
    """Phi at the points (px, py, pz) of the particles (x, y, z, w),
    truncated at lmax: the double sum written out over particles, l and m
    (a point at a particle's radius counts that particle as inside)."""
    px, py, pz = (np.atleast_1d(np.asarray(a, dtype=np.float64)) for a in (px, py, pz))
    x, y, z, w = (np.asarray(a, dtype=np.float64) for a in (x, y, z, w))
    Yp = real_harmonics(lmax, px, py, pz)
    Yi = real_harmonics(lmax, x, y, z)
    rp = np.sqrt(px * px + py * py + pz * pz)
    ri = np.sqrt(x * x + y * y + z * z)
    out = np.zeros(px.shape[0])
    for j in range(px.shape[0]):
        rl = np.minimum(rp[j], ri)
        rg = np.maximum(rp[j], ri)
        rg = np.where(rg > 0, rg, 1.0)
        acc = np.zeros_like(ri)
        for k, (l, m) in enumerate(index(lmax)):
            acc += 4 * math.pi / (2 * l + 1) * Yp[k, j] * Yi[k] * rl ** l / rg ** (l + 1)
        out[j] = -np.sum(w * acc)
    return out


# --------------------------------------------------------------------------
# The same expansion tabulated on radial nodes, as the step's axisymmetric
# expansion (:mod:`oracle.sh`) does for m = 0 and even l: the blueprint of a
# non-axisymmetric kernel.
#   A_lm(k) = sum_(r_i < r_k)          w_i r_i^l     Y_lm(x_i^),
#   B_lm(k) = sum_(r_k <= r_i < rmax)  w_i r_i^-(l+1) Y_lm(x_i^),
#   F_lm(k) = 4 pi/(2l+1) [A_lm(k) / r_k^(l+1) + B_lm(k) r_k^l],
#   D_lm(k) = 4 pi/(2l+1) [-(l+1) A_lm(k) / r_k^(l+2) + l B_lm(k) r_k^(l-1)],
#   Phi(x) = - sum_lm Y_lm(x^) F_lm(r),
# sides by r^2 in the state precision against float64 r_k^2, F and D linear
# in r between nodes, the exterior and interior laws outside them.
# --------------------------------------------------------------------------
def coefficients_nodes(x, y, z, w, rn, lmax, terms=None):
    """A_lm(r_k), B_lm(r_k), shape ((lmax+1)^2, K) (one row per term when
    `terms` is given)."""
    from . import sh as _sh
    K = len(rn)
    j = _sh.node_side(x, y, z, rn)
    keep = j < K
    xd, yd, zd = (np.asarray(v, dtype=np.float64)[keep] for v in (x, y, z))
    w = np.asarray(w, dtype=np.float64)[keep]
    j = j[keep]
    r = np.sqrt(xd * xd + yd * yd + zd * zd)
    rs = np.where(r > 0, r, 1.0)
    Y = real_harmonics(lmax, xd, yd, zd)[_rows(lmax, terms)]
    A = np.zeros((Y.shape[0], K))
    B = np.zeros((Y.shape[0], K))
    for n, (l, m) in enumerate(terms or index(lmax)):
        ta = np.bincount(j, weights=w * Y[n] * r ** l, minlength=K)
        tb = np.bincount(j, weights=np.where(j > 0, w * Y[n] * rs ** (-(l + 1)), 0.0), minlength=K)
        A[n] = np.cumsum(ta)
        B[n, :-1] = np.cumsum(tb[:0:-1])[::-1]
    return A, B


def tables_nodes(A, B, rn, lmax, terms=None):
    """F_lm(k), D_lm(k) with the 4 pi/(2l+1) of the addition theorem."""
    F = np.zeros_like(A)
    D = np.zeros_like(A)
    for n, (l, m) in enumerate(terms or index(lmax)):
        c = 4 * math.pi / (2 * l + 1)
        F[n] = c * (A[n] / rn ** (l + 1) + B[n] * rn ** l)
        D[n] = c * (-(l + 1) * A[n] / rn ** (l + 2) + (l * B[n] * rn ** (l - 1) if l > 0 else 0.0))
    return F, D


def radial_nodes(F, D, rn, r, lmax, terms=None):
    """F_lm(r), D_lm(r): linear between nodes; beyond r_(K-1)
    F(K-1) (r_(K-1)/r)^(l+1); inside r_0 F(0) (r/r_0)^l and
    D(0) (r/r_0)^max(l-1, 1)."""
    r = np.asarray(r, np.float64)
    K = len(rn)
    rc = np.clip(r, rn[0], rn[-1])
    k = np.clip(np.searchsorted(rn, rc, side="right") - 1, 0, K - 2)
    t = (rc - rn[k]) / (rn[k + 1] - rn[k])
    Fr = F[:, k] * (1 - t) + F[:, k + 1] * t
    Dr = D[:, k] * (1 - t) + D[:, k + 1] * t
    ls = np.array([l for l, _ in (terms or index(lmax))], np.float64)[:, None]
    out = r >= rn[-1]
    ro = np.where(out, r, rn[-1])
    Fo = F[:, -1:] * (rn[-1] / ro) ** (ls + 1)
    Fr = np.where(out, Fo, Fr)
    Dr = np.where(out, -(ls + 1) * Fo / ro, Dr)
    inn = r < rn[0]
    q = np.where(inn, r, rn[0]) / rn[0]
    Fr = np.where(inn, F[:, :1] * q ** ls, Fr)
    Dr = np.where(inn, D[:, :1] * q ** np.maximum(ls - 1, 1), Dr)
    return Fr, Dr


def potential_nodes(px, py, pz, F, D, rn, lmax, terms=None):
    """Phi of the tabulated expansion at the points (px, py, pz)."""
    px, py, pz = (np.atleast_1d(np.asarray(a, dtype=np.float64)) for a in (px, py, pz))
    r = np.sqrt(px * px + py * py + pz * pz)
    Y = real_harmonics(lmax, px, py, pz)[_rows(lmax, terms)]
    return -np.sum(Y * radial_nodes(F, D, rn, r, lmax, terms)[0], axis=0)


def _q_table(lmax, mu):
    """Q_l^m(mu) = d^m P_l / dmu^m for 0 <= m <= l + 1 <= lmax + 1 (zero
    when m > l): P_l^m = (1 - mu^2)^(m/2) Q_l^m, the same recurrences as
    :func:`assoc_legendre` started from Q_m^m = (2m-1)!!."""
    mu = np.asarray(mu, dtype=np.float64)
    Q = {}
    qmm = np.ones_like(mu)
    for m in range(lmax + 1):
        if m > 0:
            qmm = qmm * (2 * m - 1)
        Q[(m, m)] = qmm
        if m + 1 <= lmax:
            Q[(m + 1, m)] = (2 * m + 1) * mu * qmm
        for l in range(m + 2, lmax + 1):
            Q[(l, m)] = ((2 * l - 1) * mu * Q[(l - 1, m)] - (l + m - 1) * Q[(l - 2, m)]) / (l - m)
    zero = np.zeros_like(mu)
    return lambda l, m: Q[(l, m)] if m <= l else zero


def acceleration_nodes(px, py, pz, F, D, rn, lmax, terms=None):
    """-grad Phi of the tabulated expansion at (px, py, pz), shape (3, n).

    Written with terms that stay regular on the z axis:
      Y_lm(x) = c_lm Q_l^|m|(z/r) C_m(x, y) / r^|m|,
    C_m = Re (x + i y)^m (m >= 0) or Im (x + i y)^|m| (m < 0), c_lm = N_l0
    or sqrt(2) N_l|m|; then with n = x/r and mu = z/r
      grad Y_lm = c_lm / r^|m| [Q_l^(|m|+1) C (e_z - mu n) / r
                                + Q_l^|m| grad C - |m| Q_l^|m| C n / r],
    grad Phi = -sum_lm [D_lm(r) Y_lm n + F_lm(r) grad Y_lm]; 0 at r = 0."""
    px, py, pz = (np.atleast_1d(np.asarray(a, dtype=np.float64)) for a in (px, py, pz))
    r = np.sqrt(px * px + py * py + pz * pz)
    rs = np.where(r > 0, r, 1.0)
    n = np.stack([px, py, pz]) / rs
    mu = pz / rs
    Q = _q_table(lmax + 1, mu)
    Fr, Dr = radial_nodes(F, D, rn, r, lmax, terms)
    u = px + 1j * py
    g = np.zeros((3,) + px.shape)
    ez = np.array([0.0, 0.0, 1.0])[:, None]
    for k, (l, m) in enumerate(terms or index(lmax)):
        am = abs(m)
        N = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
        c = N if m == 0 else math.sqrt(2.0) * N
        f = u ** am
        gm = u ** (am - 1) if am > 0 else 0 * u
        if m >= 0:
            C = f.real
            dC = np.stack([am * gm.real, -am * gm.imag, 0 * px])
        else:
            C = f.imag
            dC = np.stack([am * gm.imag, am * gm.real, 0 * px])
        rm = rs ** am
        q0, q1 = Q(l, am), Q(l, am + 1)
        Y = c * q0 * C / rm
        gY = c / rm * (q1 * C * (ez - mu * n) / rs + q0 * dC - am * q0 * C * n / rs)
        g += -(Dr[k] * Y * n + Fr[k] * gY)
    return np.where(r > 0, -g, 0.0)


# --------------------------------------------------------------------------
# The triaxial expansion of the step (potential kind 'sh_tri', parameters
# (K, rmin, rmax, period)): the terms of :func:`triaxial_terms` at lmax = 8
# tabulated on the nodes of :func:`oracle.sh.nodes`, recomputed from the
# particles every `period` steps like the axisymmetric expansion.
# --------------------------------------------------------------------------
LMAX_TRI = 8


def tri_tables(x, y, z, w, rn):
    """(F, D, rn) of the triaxial expansion of the weighted particles."""
    terms = triaxial_terms(LMAX_TRI)
    A, B = coefficients_nodes(x, y, z, w, rn, LMAX_TRI, terms)
    F, D = tables_nodes(A, B, rn, LMAX_TRI, terms)
    return F, D, rn


def tri_acceleration(x, y, z, F, D, rn):
    return acceleration_nodes(x, y, z, F, D, rn, LMAX_TRI, triaxial_terms(LMAX_TRI))


def tri_potential(x, y, z, F, D, rn):
    return potential_nodes(x, y, z, F, D, rn, LMAX_TRI, triaxial_terms(LMAX_TRI))


# --------------------------------------------------------------------------
# The general expansion of the step (potential kind 'sh_full', parameters
# (K, rmin, rmax, period)): every term of :func:`index` up to l = 4 (25
# terms, cosine and sine harmonics), for models with no symmetry, on the
# same nodes and schedule.
# --------------------------------------------------------------------------
LMAX_FULL = 4


def full_tables(x, y, z, w, rn):
    """(F, D, rn) of the general expansion (l <= 4) of the weighted particles."""
    A, B = coefficients_nodes(x, y, z, w, rn, LMAX_FULL)
    F, D = tables_nodes(A, B, rn, LMAX_FULL)
    return F, D, rn


def full_acceleration(x, y, z, F, D, rn):
    return acceleration_nodes(x, y, z, F, D, rn, LMAX_FULL)


def full_potential(x, y, z, F, D, rn):
    return potential_nodes(x, y, z, F, D, rn, LMAX_FULL)

