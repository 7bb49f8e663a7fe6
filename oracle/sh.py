"""Self-consistent potential by a spherical-harmonic expansion (oracle; test
infrastructure only).

The paper notes that the potential the particles orbit in may also be
derived from the particles themselves (Section 1) and updated while the
weights adapt (Section 2).  Reading used here: the
axisymmetric (m = 0) multipole expansion of the weighted particles with even
l = 0, 2, ..., 8, G = 1:

  Phi(r, theta) = - sum_l P_l(mu) [A_l(r) / r^(l+1) + B_l(r) r^l],  mu = cos theta,
  A_l(r) = sum_{i: r_i < r}          w_i P_l(mu_i) r_i^l,
  B_l(r) = sum_{i: r <= r_i < rmax}  w_i P_l(mu_i) r_i^-(l+1),

evaluated at K radial nodes r_k = rmin (rmax/rmin)^(k/(K-1)) (so r_(K-1) =
rmax).  Which side of a node a particle lies on is decided, like the shell
membership of the observables, by its r^2 = (x*x + y*y) + z*z in the state
precision against the float64 squares r_k^2 (half-open: r^2 < r_k^2 counts in
A_l(r_k)); the terms themselves are float64 functions of the position.  Node
tables

  F_l(k) = A_l(r_k)/r_k^(l+1) + B_l(r_k) r_k^l,
  D_l(k) = -(l+1) A_l(r_k)/r_k^(l+2) + l B_l(r_k) r_k^(l-1)   (= dF_l/dr, the
           terms from dA/dr and dB/dr cancel),

are interpolated linearly in r between nodes:  Phi = -sum P_l F_l(r),
dPhi/dr = -sum P_l D_l(r), dPhi/dmu = -sum P_l'(mu) F_l(r), a = -grad Phi.
Outside the nodes:
  r >= r_(K-1): the exterior law F_l(r) = F_l(K-1) (r_(K-1)/r)^(l+1),
                D_l(r) = -(l+1) F_l(r)/r, exact because every particle that
                is counted lies inside rmax;
  r <  r_0:     F_l(r) = F_l(0) (r/r_0)^l, D_l(r) = D_l(0) (r/r_0)^max(l-1, 1):
                the interior solution for l >= 2 and a uniform core for
                l = 0, so F and D stay continuous and the force falls to 0
                at the centre.
At r = 0 the acceleration is 0.
"""
import numpy as np

LS = (0, 2, 4, 6, 8)


def legendre(mu, lmax=8):
    """P_0..P_lmax by Bonnet's recurrence, shape (lmax+1, ...)."""
    mu = np.asarray(mu, dtype=np.float64)
    P = [np.ones_like(mu), mu.copy()]
    for l in range(1, lmax):
        P.append(((2 * l + 1) * mu * P[l] - l * P[l - 1]) / (l + 1))
    return np.stack(P[:lmax + 1])


def legendre_deriv(mu, lmax=8):
    """P'_0..P'_lmax via P'_(l+1) = P'_(l-1) + (2l+1) P_l."""
    P = legendre(mu, lmax)
    D = [np.zeros_like(P[0]), np.ones_like(P[0])]
    for l in range(1, lmax):
        D.append(D[l - 1] + (2 * l + 1) * P[l])
    return np.stack(D[:lmax + 1])


def nodes(rmin, rmax, K):
    k = np.arange(K, dtype=np.float64)
    rn = rmin * (rmax / rmin) ** (k / (K - 1))
    rn[-1] = rmax
    return rn


def node_side(x, y, z, rn):
    """j_i = number of nodes with r_k^2 <= r_i^2 (r^2 in the state precision,
    compared in float64); a particle counts in A_l(r_k) for k >= j_i and in
    B_l(r_k) for k < j_i.  j_i = K means r_i >= rmax: left out."""
    r2 = (x * x + y * y) + z * z
    e = np.asarray(rn, np.float64) ** 2
    j = np.searchsorted(e, np.asarray(r2).astype(np.float64), side="right")
    return np.where(np.isnan(r2), len(rn), j)


def coefficients(x, y, z, w, rn):
    """A_l(r_k), B_l(r_k) for l in LS, shape (5, K): per-side sums by
    bincount, then a prefix sum (A) and a suffix sum (B) over the sides."""
    K = len(rn)
    j = node_side(x, y, z, rn)
    xd, yd, zd = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    w = np.asarray(w, dtype=np.float64)
    r = np.sqrt(xd * xd + yd * yd + zd * zd)
    keep = j < K
    j, r, zd, w = j[keep], r[keep], zd[keep], w[keep]
    rs = np.where(r > 0, r, 1.0)
    mu = np.where(r > 0, zd / rs, 0.0)
    P = legendre(mu)
    A = np.zeros((len(LS), K))
    B = np.zeros((len(LS), K))
    for n, l in enumerate(LS):
        ta = np.bincount(j, weights=w * P[l] * r ** l, minlength=K)
        # side 0 (r < r_0, r = 0 included) never counts in B: leave it out
        # rather than subtract it, since its terms r^-(l+1) can be huge
        tb = np.bincount(j, weights=np.where(j > 0, w * P[l] * rs ** (-(l + 1)), 0.0),
                         minlength=K)
        A[n] = np.cumsum(ta)                        # sides j <= k
        B[n, :-1] = np.cumsum(tb[:0:-1])[::-1]      # sides j > k, summed outside in
    return A, B


def tables(A, B, rn):
    """F_l(k), D_l(k), shape (5, K)."""
    F = np.zeros_like(A)
    D = np.zeros_like(A)
    for n, l in enumerate(LS):
        F[n] = A[n] / rn ** (l + 1) + B[n] * rn ** l
        D[n] = -(l + 1) * A[n] / rn ** (l + 2) + (l * B[n] * rn ** (l - 1) if l > 0 else 0.0)
    return F, D


def radial(F, D, rn, r):
    """F_l(r), D_l(r) at radii r (interpolated, or the laws outside)."""
    r = np.asarray(r, np.float64)
    K = len(rn)
    rc = np.clip(r, rn[0], rn[-1])
    k = np.clip(np.searchsorted(rn, rc, side="right") - 1, 0, K - 2)
    t = (rc - rn[k]) / (rn[k + 1] - rn[k])
    Fr = F[:, k] * (1 - t) + F[:, k + 1] * t
    Dr = D[:, k] * (1 - t) + D[:, k + 1] * t
    ls = np.asarray(LS, np.float64)[:, None]
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


def potential(x, y, z, F, D, rn):
    xd, yd, zd = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    r = np.sqrt(xd * xd + yd * yd + zd * zd)
    mu = np.where(r > 0, zd / np.where(r > 0, r, 1.0), 0.0)
    P = legendre(mu)[list(LS)]
    return -np.sum(P * radial(F, D, rn, r)[0], axis=0)


def acceleration(x, y, z, F, D, rn):
    """-grad Phi of the interpolated expansion, float64, shape 3 x (...)."""
    xd, yd, zd = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    r = np.sqrt(xd * xd + yd * yd + zd * zd)
    rs = np.where(r > 0, r, 1.0)
    mu = zd / rs
    P = legendre(mu)[list(LS)]
    dP = legendre_deriv(mu)[list(LS)]
    Fr, Dr = radial(F, D, rn, r)
    dphi_dr = -np.sum(P * Dr, axis=0)
    dphi_dmu = -np.sum(dP * Fr, axis=0)
    # mu = z/r: dmu/dx = -z x / r^3, dmu/dy = -z y / r^3, dmu/dz = (x^2+y^2) / r^3
    r3 = rs ** 3
    gx = dphi_dr * xd / rs + dphi_dmu * (-zd * xd / r3)
    gy = dphi_dr * yd / rs + dphi_dmu * (-zd * yd / r3)
    gz = dphi_dr * zd / rs + dphi_dmu * ((xd * xd + yd * yd) / r3)
    zero = r == 0
    return (np.where(zero, 0.0, -gx), np.where(zero, 0.0, -gy), np.where(zero, 0.0, -gz))
