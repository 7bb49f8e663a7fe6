"""Gauss-Hermite line-of-sight kernels (oracle; test infrastructure only).

The paper lists integral-field absorption-line kinematics among the data the
weights are fitted to (Section 1).  Those data are Gauss-Hermite moments
h_n of the line-of-sight velocity distribution in the normalisation of
van der Marel & Franx (1993): with w = (v - V)/S,

    alpha(w) = exp(-w^2/2) / sqrt(2 pi),
    h_n      = 2 sqrt(pi) * integral L(v) alpha(w) H_n(w) dv,

so a unit Gaussian with the reference V, S has h0 = 1, h1..h4 = 0.  For
particles, L(v) is a sum of weighted spikes smoothed by a Gaussian velocity
kernel of width sigma_k; the particle's contribution per unit weight is

    u_n(nu) = 2 sqrt(pi) E_{nu' ~ N(nu, s^2)} [alpha(nu') H_n(nu')],
    nu = (v_los - V)/S,  s = sigma_k / S.

Completing the square, alpha(nu') N(nu'; nu, s^2) = N(nu; 0, 1+s^2) N(nu'; m, t2)
with m = nu/(1+s^2), t2 = s^2/(1+s^2), so u_n is a Gaussian factor times the
expectation of a polynomial, which only needs raw Gaussian moments up to 4.
"""
import math

import numpy as np

SQRT2 = math.sqrt(2.0)
SQRT3 = math.sqrt(3.0)
SQRT24 = math.sqrt(24.0)
TWO_SQRT_PI = 2.0 * math.sqrt(math.pi)


def hermite(y):
    """H_0..H_4 of van der Marel & Franx (1993), shape (..., 5)."""
    y = np.asarray(y, dtype=np.float64)
    H0 = np.ones_like(y)
    H1 = SQRT2 * y
    H2 = (2.0 * y * y - 1.0) / SQRT2
    H3 = (2.0 * y ** 3 - 3.0 * y) / SQRT3
    H4 = (4.0 * y ** 4 - 12.0 * y * y + 3.0) / SQRT24
    return np.stack([H0, H1, H2, H3, H4], axis=-1)


def alpha(y):
    y = np.asarray(y, dtype=np.float64)
    return np.exp(-0.5 * y * y) / math.sqrt(2.0 * math.pi)


def gh_point(nu):
    """Unsmoothed kernel u_n = 2 sqrt(pi) alpha(nu) H_n(nu), shape (..., 5)."""
    nu = np.asarray(nu, dtype=np.float64)
    return TWO_SQRT_PI * alpha(nu)[..., None] * hermite(nu)


def gh_kernel(nu, s):
    """Gaussian-smoothed kernel u_n(nu; s), n = 0..4, shape (..., 5).

    nu, s broadcast; s = 0 gives :func:`gh_point`.
    """
    nu = np.asarray(nu, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    d = 1.0 + s * s
    m = nu / d
    t2 = s * s / d
    gauss = np.exp(-0.5 * nu * nu / d) / np.sqrt(2.0 * math.pi * d)
    E1 = m
    E2 = m * m + t2
    E3 = m ** 3 + 3.0 * m * t2
    E4 = m ** 4 + 6.0 * m * m * t2 + 3.0 * t2 * t2
    EH = np.stack([np.ones_like(E1 * 1.0 + 0 * t2),
                   SQRT2 * E1,
                   (2.0 * E2 - 1.0) / SQRT2,
                   (2.0 * E3 - 3.0 * E1) / SQRT3,
                   (4.0 * E4 - 12.0 * E2 + 3.0) / SQRT24], axis=-1)
    return TWO_SQRT_PI * gauss[..., None] * EH
