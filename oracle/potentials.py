"""Analytic potentials and accelerations (oracle; test infrastructure only).

The particles are evolved in a gravitational potential that is fixed and
known (Section 2, after Eq. 2).  G = 1.  The potential is a sum of
components; each component is (kind, params):

  'hernquist' (GM, a):     Phi = -GM/(r+a),   a(x) = -GM x / (r (r+a)^2)
  'nfw'       (rho_s, r_s): Phi = -4 pi rho_s r_s^3 ln(1+r/r_s)/r,
                            a(x) = -M(r) x / r^3,
                            M(r) = 4 pi rho_s r_s^3 [ln(1+u) - u/(1+u)], u=r/r_s
  'log'       (v0, Rc, q): Phi = 1/2 v0^2 ln(D), D = Rc^2 + x^2 + y^2 + z^2/q^2,
                            a = -v0^2 (x, y, z/q^2) / D

Evaluation order (it decides rounding, and positions feed integer bin
decisions, so it is fixed here and in the kernels alike):

  hernquist: r2 = (x*x + y*y) + z*z;  r = sqrt(r2);  s = r + a;
             f = GM / ((r*s)*s)   (f = 0 where r2 == 0);  a_k = -(f*x_k)
  log:       R2 = x*x + y*y;  D = (Rc2 + R2) + (z*z)*iq2;  f = v0sq / D;
             a_x = -(f*x), a_y = -(f*y), a_z = -((f*iq2)*z)
  nfw:       f = M(r)/r^3 evaluated in float64 from the stored position,
             then rounded to the state precision; a_k = -(f*x_k)

The derived constants (Rc2 = Rc*Rc, iq2 = 1/(q*q), v0sq = v0*v0) are formed
in float64 and rounded once to the state precision.  Components are summed in
the order given, starting from zero.
"""
import math

import numpy as np

from .flog import log_f32, log_f64


def _cast(T, v):
    return np.asarray(v, dtype=np.float64).astype(T)


def _nfw_f(r, rho_s, r_s):
    """M(r)/r^3 in float64 (series for small u)."""
    r = np.asarray(r, dtype=np.float64)
    u = r / r_s
    small = u < 1e-3
    us = np.where(small, 1.0, u)
    big = np.log1p(us) - us / (1.0 + us)
    ser = u * u * (0.5 - u * (2.0 / 3.0 - u * (0.75 - 0.8 * u)))
    mu = np.where(small, ser, big)
    rr = np.where(r > 0, r, 1.0)
    f = 4.0 * math.pi * rho_s * r_s ** 3 * mu / (rr ** 3)
    # limit r -> 0: M ~ 2 pi rho_s r_s r^2 so f ~ 2 pi rho_s r_s / r; the
    # acceleration f*x stays finite (|a| -> 2 pi rho_s r_s); define f=0 at r=0
    return np.where(r > 0, f, 0.0)


def acceleration(x, y, z, comps):
    """Acceleration (ax, ay, az) in the dtype of x, y, z."""
    T = x.dtype.type
    ax = np.zeros_like(x)
    ay = np.zeros_like(x)
    az = np.zeros_like(x)
    with np.errstate(divide="ignore", invalid="ignore"):
        for c in comps:
            if c.kind == "hernquist":
                GM, a = _cast(T, c.params[0]), _cast(T, c.params[1])
                r2 = (x * x + y * y) + z * z
                r = np.sqrt(r2)
                s = r + a
                f = np.where(r2 > 0, GM / ((r * s) * s), T(0))
                ax = ax + (-(f * x))
                ay = ay + (-(f * y))
                az = az + (-(f * z))
            elif c.kind == "log":
                v0, Rc, q = c.params
                Rc2 = _cast(T, Rc * Rc)
                iq2 = _cast(T, 1.0 / (q * q))
                v0sq = _cast(T, v0 * v0)
                R2 = x * x + y * y
                D = (Rc2 + R2) + (z * z) * iq2
                f = v0sq / D
                ax = ax + (-(f * x))
                ay = ay + (-(f * y))
                az = az + (-((f * iq2) * z))
            elif c.kind == "nfw":
                rho_s, r_s = c.params
                xd, yd, zd = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
                r = np.sqrt(xd * xd + yd * yd + zd * zd)
                f = _nfw_f(r, rho_s, r_s).astype(T)
                ax = ax + (-(f * x))
                ay = ay + (-(f * y))
                az = az + (-(f * z))
            elif c.kind == "sh":
                raise ValueError("the spherical-harmonic component needs the particles: use oracle.m2m")
            else:
                raise ValueError(f"unknown potential kind {c.kind!r}")
    return ax, ay, az


def potential(x, y, z, comps):
    """Potential Phi in the dtype of x, y, z (used for the prior cells).

    hernquist: r2 = (x*x + y*y) + z*z; Phi = -(GM / (sqrt(r2) + a))
    log:       Phi = (0.5*v0sq) * ln(D), D as in :func:`acceleration`; ln
               is :func:`oracle.flog.log_f32` / :func:`oracle.flog.log_f64`
               (fixed sequences of float32 / float64 operations, so that the
               prior cells do not depend on a library's rounding of the
               logarithm)
    nfw:       float64 evaluation rounded to the state precision
    """
    T = x.dtype.type
    phi = np.zeros_like(x)
    with np.errstate(divide="ignore", invalid="ignore"):
        for c in comps:
            if c.kind == "hernquist":
                GM, a = _cast(T, c.params[0]), _cast(T, c.params[1])
                r2 = (x * x + y * y) + z * z
                phi = phi + (-(GM / (np.sqrt(r2) + a)))
            elif c.kind == "log":
                v0, Rc, q = c.params
                Rc2 = _cast(T, Rc * Rc)
                iq2 = _cast(T, 1.0 / (q * q))
                hv = _cast(T, 0.5 * v0 * v0)
                R2 = x * x + y * y
                D = (Rc2 + R2) + (z * z) * iq2
                # the fixed-order logarithm of oracle.flog in the state
                # precision, which the GPU path evaluates identically
                phi = phi + hv * (log_f32(D) if T is np.float32 else log_f64(D))
            elif c.kind == "nfw":
                rho_s, r_s = c.params
                xd, yd, zd = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
                r = np.sqrt(xd * xd + yd * yd + zd * zd)
                u = r / r_s
                rr = np.where(r > 0, r, 1.0)
                ph = np.where(r > 0, -4.0 * math.pi * rho_s * r_s ** 3 * np.log1p(u) / rr,
                              -4.0 * math.pi * rho_s * r_s ** 2)
                phi = phi + ph.astype(T)
            else:
                raise ValueError(f"unknown potential kind {c.kind!r}")
    return phi
