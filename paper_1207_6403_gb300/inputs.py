"""Seeded synthetic inputs for the made-to-measure (M2M) training step.

This module is shared by the CUDA path and by the test oracle, so it holds
none of the M2M step's own arithmetic: no orbit push, no bin membership, no
observable kernel, no residual, weight update or prior.  It only

* draws particle realisations (initial models and target galaxies) from
  Philox-seeded numpy generators (Salmon et al. 2011 counter-based RNG);
* builds the bin-edge tables that *define* the observables (squared radii for
  3D shells and projected annuli, x/y edges for pixel and aperture grids);
* fixes the per-aperture Gauss-Hermite reference velocity and width;
* states the observational error model sigma_j (2% of the target value);
* describes each workload as plain data (:class:`Problem`).

The target observables Y_j are *not* produced here: a caller observes the
target realisation with whichever implementation it trusts (the oracle in the
tests, the library itself when timing), then applies :func:`error_model`.

Physical units: G = 1 throughout.  The workloads follow the paper's problem
statement (Section 2: particles with weights w_i in a potential, observables
with errors, priors w_hat_i; Section 2.1: flat priors 1/N and moving priors
in integral-of-motion space) at the sizes of the five benchmark workloads:

  plain-fp64    N=20,000 Hernquist, 40 shells + 20 annuli (mass, v_los^2), FP64
  moving-priors N=1,000,000 Hernquist, 100 shells + 60 annuli x h0..h4, (E, L^2/Lc^2) priors
  flat-log      N=4,000,000 flattened logarithmic potential at 60 deg, 64x64 pixels +
                20x20 apertures x h0..h4, (E, L_z) priors
  batched       48 Hernquist+NFW models, N log-uniform in [1e5, 2e6], halo grid
                (M_h/M_*, r_s/a) of 6 x 8, each with its own targets (make_batch)
  sh-selfcons   N=8,000,000 Miyamoto-Nagai disc + Hernquist bulge (1:3) moving in
                the spherical-harmonic expansion of their own weighted mass,
                recomputed every 50 steps; observables as moving-priors, flat priors
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

__all__ = [
    "PotentialComponent", "ObservableSet", "PriorSpec", "Problem",
    "rng", "hernquist_positions", "hernquist_isotropic", "hernquist_om_target",
    "log_flattened_realisation", "log_shell_edges", "uniform_edges",
    "error_model", "make_problem", "make_batch", "make_scan", "WORKLOADS", "disc_bulge_realisation",
]


# --------------------------------------------------------------------------
# Plain-data workload description
# --------------------------------------------------------------------------
@dataclass
class PotentialComponent:
    """One analytic potential component; the potential is the sum of them.

    kind 'hernquist': params (GM, a)           Phi = -GM/(r+a)
    kind 'nfw':       params (rho_s, r_s)      Phi = -4 pi rho_s r_s^3 ln(1+r/r_s)/r
    kind 'log':       params (v0, Rc, q)       Phi = 1/2 v0^2 ln(Rc^2 + R^2 + z^2/q^2)
    kind 'sh':        params (K, rmin, rmax, period)
                      the potential of the weighted particles themselves,
                      expanded in even Legendre multipoles l <= 8 on K
                      log-spaced radial nodes in [rmin, rmax] and recomputed
                      every `period` steps (at most one, listed last)
    """
    kind: str
    params: tuple


@dataclass
class ObservableSet:
    """One set of observables y_j = sum_i w_i K_j(x_i, v_i).

    geom  'shell'   : cells are 3D radial shells, edges_x are edges of r^2
          'annulus' : cells are projected annuli, edges_x are edges of R^2
          'grid'    : cells are rectangles of the sky plane (pixels or IFU
                      apertures), edges_x / edges_y are edges of X / Y
          'lut'     : cells are sky apertures of any shape (Voronoi bins,
                      long-slit segments): the sky pixel (ix, iy) by edges_x /
                      edges_y as for 'grid', then cell = lut[iy, ix] (-1: no
                      cell); n_apertures cells
    quant 'mass'    : K = 1 in the cell
          'vlos2'   : K = v_los^2 in the cell (luminosity-weighted 2nd moment)
          'gh'      : K_n = Gauss-Hermite kernel u_n, n = 0..4, in the cell,
                      about (gh_V, gh_S) per cell, convolved with a Gaussian
                      velocity kernel of width sigma_kernel
    Cell index: grid cell = iy * nx + ix.  Observable index inside the set =
    cell * nmom + n.  Edge arrays are float64 and strictly increasing; the
    membership of a value v in cell j is e_j <= v < e_{j+1}.
    """
    geom: str
    quant: str
    edges_x: np.ndarray
    edges_y: Optional[np.ndarray] = None
    gh_V: Optional[np.ndarray] = None
    gh_S: Optional[np.ndarray] = None
    sigma_kernel: float = 0.0
    lut: Optional[np.ndarray] = None       # 'lut': (ny, nx) int32 cell ids
    n_apertures: int = 0                   # 'lut': number of cells
    # seeing (projected sets): 2^b displacement quantiles of the PSF along
    # one sky axis, and the key of the counter-based draws
    psf_q: Optional[np.ndarray] = None
    psf_seed: int = 0

    @property
    def nx(self) -> int:
        return len(self.edges_x) - 1

    @property
    def ny(self) -> int:
        return 1 if self.edges_y is None else len(self.edges_y) - 1

    @property
    def ncells(self) -> int:
        return self.n_apertures if self.geom == "lut" else self.nx * self.ny

    @property
    def nmom(self) -> int:
        return 5 if self.quant == "gh" else 1

    @property
    def nobs(self) -> int:
        return self.ncells * self.nmom


@dataclass
class PriorSpec:
    """How the priors w_hat_i are set (Section 2.1).

    kind 'flat' : w_hat_i stay at their initial value (1/N).
    kind 'e_lc' : every `period` steps, w_hat_i = mean weight of the particles
                  in i's cell of an nE x nL grid in (E, L^2/Lc^2(E)) for a
                  Hernquist potential (GM, a) = hernquist; E-cells are uniform
                  on [min E, 0), unbound particles share one extra cell.
    kind 'e_lz' : the same on an nE x nL grid in (E, L_z), uniform on
                  [min E, max E] x [-max|L_z|, max|L_z|].
    kind 'e_l2' : the same on an nE x nL grid in (E, L^2), uniform on
                  [min E, max E] x [0, max L^2] (potentials without a
                  symmetry axis).
    """
    kind: str = "flat"
    nE: int = 1
    nL: int = 1
    period: int = 25
    hernquist: tuple = (1.0, 1.0)

    @property
    def ncells(self) -> int:
        if self.kind == "flat":
            return 0
        return self.nE * self.nL + (1 if self.kind == "e_lc" else 0)


@dataclass
class Problem:
    """A complete M2M workload as plain arrays and numbers."""
    name: str
    n: int
    pos: np.ndarray            # (3, n) float64
    vel: np.ndarray            # (3, n) float64
    w0: np.ndarray             # (n,) float64
    what0: np.ndarray          # (n,) float64
    potential: List[PotentialComponent]
    obs: List[ObservableSet]
    incl_sin: float            # line of sight s = (0, sin i, cos i)
    incl_cos: float
    eps: float                 # effective epsilon (the workload's epsilon / N)
    mu: float
    dt: float
    alpha: float
    prior: PriorSpec
    nsteps: int
    precision: str             # 'fp64' or 'fp32c'
    entropy_const: float = 1.0  # dS/dw_i = -ln(w_i/w_hat_i) - entropy_const
    target_pos: Optional[np.ndarray] = None
    target_vel: Optional[np.ndarray] = None
    target_w: Optional[np.ndarray] = None
    Y: Optional[np.ndarray] = None
    sigma: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def nobs(self) -> int:
        return sum(s.nobs for s in self.obs)

    def with_targets(self, Y: np.ndarray) -> "Problem":
        """Return a copy carrying targets Y and the 2% error model."""
        Y = np.asarray(Y, dtype=np.float64)
        return replace(self, Y=Y, sigma=error_model(Y, self.obs))


# --------------------------------------------------------------------------
# Random streams
# --------------------------------------------------------------------------
def rng(seed: int) -> np.random.Generator:
    """Philox4x32-10 counter-based stream (Salmon et al. 2011) for one seed."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _isotropic_directions(g: np.random.Generator, n: int):
    cth = g.uniform(-1.0, 1.0, n)
    phi = g.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return sth * np.cos(phi), sth * np.sin(phi), cth


# --------------------------------------------------------------------------
# Hernquist model (Hernquist 1990, ApJ 356, 359), G = 1
# --------------------------------------------------------------------------
def _hernquist_rho(r, M=1.0, a=1.0):
    return M * a / (2.0 * math.pi * r * (r + a) ** 3)


def _hernquist_mass(r, M=1.0, a=1.0):
    return M * r * r / ((r + a) ** 2)


def _jeans_sigma_r2_table(rho, mass, ra=None, rmin=1e-5, rmax=1e4, npts=480, beta=None):
    """sigma_r^2(r) on a log grid from the spherical Jeans equation.

    Isotropic (ra None):  rho sigma^2 = int_r^inf rho M / r'^2 dr'.
    Osipkov-Merritt-like beta = r^2/(r^2+ra^2):
        rho (r^2+ra^2) sigma_r^2 = int_r^inf (r'^2+ra^2) rho M / r'^2 dr'.
    Constant beta:  rho r^(2 beta) sigma_r^2 = int_r^inf r'^(2 beta) rho M / r'^2 dr'.
    Integrated in ln r' with composite Simpson on a fine grid plus an
    analytic r'^-4 tail beyond rmax.
    """
    lr = np.linspace(math.log(rmin), math.log(rmax), 8 * npts + 1)
    r = np.exp(lr)
    if beta is not None:
        g = r ** (2.0 * beta)
    else:
        g = np.ones_like(r) if ra is None else r * r + ra * ra
    f = g * rho(r) * mass(r) / (r * r) * r          # integrand in d ln r
    # cumulative integral from each grid point to rmax (trapezoid on a fine grid
    # is refined by Richardson with the half grid: error ~ h^4)
    h = lr[1] - lr[0]
    seg = 0.5 * h * (f[1:] + f[:-1])
    tail_fine = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    f2 = f[::2]
    seg2 = 0.5 * (2 * h) * (f2[1:] + f2[:-1])
    tail_coarse = np.concatenate([np.cumsum(seg2[::-1])[::-1], [0.0]])
    tail = (4.0 * tail_fine[::2] - tail_coarse) / 3.0
    rr = r[::2]
    # analytic continuation past rmax: integrand ~ C r'^-3 (isotropic) or r'^-1... use
    # the local power law of f to extend
    slope = (math.log(f[-1]) - math.log(f[-9])) / (lr[-1] - lr[-9])
    extra = -f[-1] / slope if slope < 0 else 0.0
    tail = tail + extra
    gg = g[::2]
    sig2 = tail / (gg * rho(rr))
    return rr, sig2


class _Interp:
    def __init__(self, r, y):
        self.lr = np.log(r)
        self.ly = np.log(np.maximum(y, 1e-300))

    def __call__(self, r):
        return np.exp(np.interp(np.log(r), self.lr, self.ly))


def hernquist_sigma_iso(GM=1.0, a=1.0):
    """Callable isotropic sigma^2(r) of a Hernquist sphere (Jeans quadrature)."""
    rr, s2 = _jeans_sigma_r2_table(lambda r: _hernquist_rho(r, GM, a),
                                   lambda r: _hernquist_mass(r, GM, a))
    return _Interp(rr, s2)


def hernquist_positions(n, seed, GM=1.0, a=1.0, rmax=100.0):
    """Positions (3, n) of a Hernquist sphere truncated at rmax, sorted by r.

    Radius by the inverse of M(<r)/M = r^2/(r+a)^2: r = a sqrt(u)/(1-sqrt(u)).
    Returns (pos, r, g) where g is the generator, so velocities come from the
    same stream.
    """
    g = rng(seed)
    umax = (rmax / (rmax + a)) ** 2
    u = g.uniform(0.0, umax, n)
    su = np.sqrt(u)
    r = a * su / (1.0 - su)
    r.sort()
    ex, ey, ez = _isotropic_directions(g, n)
    pos = np.stack([r * ex, r * ey, r * ez])
    return pos, r, g


def _spherical_gaussian_velocities(g, pos, r, sig_r, sig_t):
    """Gaussian velocities with radial / tangential dispersions (local frame)."""
    n = r.shape[0]
    vr = g.standard_normal(n) * sig_r
    vt1 = g.standard_normal(n) * sig_t
    vt2 = g.standard_normal(n) * sig_t
    rs = np.where(r > 0, r, 1.0)
    er = pos / rs
    # tangential basis: e_theta, e_phi from er
    x, y, z = er
    Rxy = np.sqrt(x * x + y * y)
    Rs = np.where(Rxy > 0, Rxy, 1.0)
    ephi = np.stack([-y / Rs, x / Rs, np.zeros_like(x)])
    eth = np.stack([z * x / Rs, z * y / Rs, -Rxy])
    return er * vr + eth * vt1 + ephi * vt2


def hernquist_isotropic(n, seed, GM=1.0, a=1.0, rmax=100.0):
    """Isotropic Hernquist realisation: positions by inverse CDF, velocities
    Gaussian with the isotropic Jeans sigma(r)."""
    pos, r, g = hernquist_positions(n, seed, GM, a, rmax)
    s2 = hernquist_sigma_iso(GM, a)(r)
    s = np.sqrt(s2)
    vel = _spherical_gaussian_velocities(g, pos, r, s, s)
    return pos, vel


def hernquist_om_target(n, seed, ra=1.0, GM=1.0, a=1.0, rmax=100.0):
    """Osipkov-Merritt-like Hernquist target: beta(r) = r^2/(r^2+ra^2),
    sigma_t = sqrt(1-beta) sigma_r, Gaussian velocities."""
    pos, r, g = hernquist_positions(n, seed, GM, a, rmax)
    rr, s2 = _jeans_sigma_r2_table(lambda x: _hernquist_rho(x, GM, a),
                                   lambda x: _hernquist_mass(x, GM, a), ra=ra)
    sr = np.sqrt(_Interp(rr, s2)(r))
    beta = r * r / (r * r + ra * ra)
    st = np.sqrt(1.0 - beta) * sr
    vel = _spherical_gaussian_velocities(g, pos, r, sr, st)
    return pos, vel


def hernquist_const_beta(n, seed, beta, GM=1.0, a=1.0, rmax=100.0):
    """Hernquist realisation with a constant anisotropy beta (< 0:
    tangential), sigma_t = sqrt(1-beta) sigma_r from the Jeans equation,
    Gaussian velocities."""
    pos, r, g = hernquist_positions(n, seed, GM, a, rmax)
    rr, s2 = _jeans_sigma_r2_table(lambda x: _hernquist_rho(x, GM, a),
                                   lambda x: _hernquist_mass(x, GM, a), beta=beta)
    sr = np.sqrt(_Interp(rr, s2)(r))
    vel = _spherical_gaussian_velocities(g, pos, r, sr, math.sqrt(1.0 - beta) * sr)
    return pos, vel


# --------------------------------------------------------------------------
# Flattened logarithmic potential (Binney & Tremaine eq. 2.71)
# --------------------------------------------------------------------------
def log_flattened_density(x, y, z, v0=1.0, Rc=0.1, q=0.8):
    """Density generating Phi = 1/2 v0^2 ln(Rc^2 + R^2 + z^2/q^2), G = 1."""
    R2 = x * x + y * y
    D = Rc * Rc + R2 + z * z / (q * q)
    num = (2 * q * q + 1) * Rc * Rc + R2 + (2 - 1 / (q * q)) * z * z
    return v0 * v0 / (4 * math.pi * q * q) * num / (D * D)


def log_flattened_realisation(n, seed, v0=1.0, Rc=0.1, q=0.8, mmax=5.0,
                              stream_frac=0.0):
    """Particles of the flattened-log density truncated at
    m = sqrt(R^2 + z^2/q^2) <= mmax, sorted by m.

    Proposal: m with density ~ m^2/(Rc^2+m^2) on [0, mmax], isotropic
    direction in ellipsoidal coordinates (x, y, z) = m (sin t cos p,
    sin t sin p, q cos t); accepted with probability rho/(proposal) divided by
    its bound (2 q^2 + 1).  Velocities isotropic Gaussian, sigma^2 = v0^2/2,
    plus an azimuthal streaming stream_frac * v_c(R),
    v_c^2 = v0^2 R^2/(Rc^2 + R^2).
    """
    g = rng(seed)
    out = []
    have = 0
    bound = 2 * q * q + 1
    while have < n:
        k = int((n - have) * 2.4) + 1024
        m = g.uniform(0.0, mmax, k)
        keep_m = g.uniform(0.0, 1.0, k) < (m * m / (Rc * Rc + m * m))
        m = m[keep_m]
        kk = m.shape[0]
        ex, ey, ez = _isotropic_directions(g, kk)
        x, y, z = m * ex, m * ey, q * m * ez
        R2 = x * x + y * y
        num = (2 * q * q + 1) * Rc * Rc + R2 + (2 - 1 / (q * q)) * z * z
        ratio = num / (Rc * Rc + m * m)
        acc = g.uniform(0.0, bound, kk) < ratio
        out.append(np.stack([x[acc], y[acc], z[acc]]))
        have += int(acc.sum())
    pos = np.concatenate(out, axis=1)[:, :n]
    mm = np.sqrt(pos[0] ** 2 + pos[1] ** 2 + (pos[2] / q) ** 2)
    order = np.argsort(mm, kind="stable")
    pos = np.ascontiguousarray(pos[:, order])
    sig = v0 / math.sqrt(2.0)
    vel = g.standard_normal((3, n)) * sig
    if stream_frac:
        R = np.sqrt(pos[0] ** 2 + pos[1] ** 2)
        vc = v0 * R / np.sqrt(Rc * Rc + R * R)
        Rs = np.where(R > 0, R, 1.0)
        vel[0] += stream_frac * vc * (-pos[1] / Rs)
        vel[1] += stream_frac * vc * (pos[0] / Rs)
    return pos, vel


# --------------------------------------------------------------------------
# Edge tables and the error model
# --------------------------------------------------------------------------
# --------------------------------------------------------------------------
# Disc + bulge: Miyamoto & Nagai (1975) disc and a Hernquist bulge, G = 1
# --------------------------------------------------------------------------
def miyamoto_nagai_rho(R, z, M=1.0, a=1.0, b=0.2):
    zeta = np.sqrt(z * z + b * b)
    s = a + zeta
    return (b * b * M / (4 * math.pi)) * (a * R * R + (a + 3 * zeta) * s * s) / (
        (R * R + s * s) ** 2.5 * zeta ** 3)


def _mn_positions(g, n, M, a, b, Rmax=30.0, zmax=30.0, nR=600, nz=400):
    """Positions drawn from the Miyamoto-Nagai density truncated at R < Rmax,
    |z| < zmax: a cell of a (log R, asinh(z/b)) grid by the cumulative mass
    of the grid, then uniform in area and height inside the cell."""
    Re = np.concatenate([[0.0], np.geomspace(1e-3, Rmax, nR)])
    ze = b * np.sinh(np.linspace(0.0, math.asinh(zmax / b), nz + 1))
    Rm = 0.5 * (Re[1:] + Re[:-1])
    zm = 0.5 * (ze[1:] + ze[:-1])
    area = math.pi * (Re[1:] ** 2 - Re[:-1] ** 2)
    mass = miyamoto_nagai_rho(Rm[:, None], zm[None, :], M, a, b) * area[:, None] * np.diff(ze)[None, :]
    cdf = np.cumsum(mass.ravel())
    cdf /= cdf[-1]
    cell = np.minimum(np.searchsorted(cdf, g.uniform(0.0, 1.0, n), side="right"), cdf.size - 1)
    iR, iz = np.divmod(cell, nz)
    R = np.sqrt(Re[iR] ** 2 + g.uniform(0.0, 1.0, n) * (Re[iR + 1] ** 2 - Re[iR] ** 2))
    z = (ze[iz] + g.uniform(0.0, 1.0, n) * (ze[iz + 1] - ze[iz])) * np.where(g.uniform(0.0, 1.0, n) < 0.5, -1.0, 1.0)
    phi = g.uniform(0.0, 2 * math.pi, n)
    return R, phi, z


def disc_bulge_realisation(n, seed, disc_frac=0.25, Md_a=1.0, Md_b=0.2, bulge_a=0.3, rmax=30.0):
    """Disc + bulge of total mass 1 (disc : bulge = 1 : 3 by default), sorted
    by radius.  Disc: Miyamoto-Nagai (a, b), v = v_c(R) e_phi + N(0, (0.1
    v_c)^2) per component, v_c from the midplane forces of both components.
    Bulge: Hernquist (a) with isotropic Gaussian velocities from the Jeans
    equation in the bulge mass plus the disc mass taken as spherical,
    M_d r^3 / (r^2 + (a+b)^2)^(3/2)."""
    Md = disc_frac
    Mb = 1.0 - Md
    nd = int(round(n * disc_frac))
    nb = n - nd
    g = rng(seed)
    R, phi, z = _mn_positions(g, nd, Md, Md_a, Md_b, Rmax=rmax, zmax=rmax)
    vc = np.sqrt(Md * R * R / (R * R + (Md_a + Md_b) ** 2) ** 1.5 + Mb * R / (R + bulge_a) ** 2)
    cp, sp = np.cos(phi), np.sin(phi)
    vR = 0.1 * vc * g.standard_normal(nd)
    vp = vc + 0.1 * vc * g.standard_normal(nd)
    vz = 0.1 * vc * g.standard_normal(nd)
    dpos = np.stack([R * cp, R * sp, z])
    dvel = np.stack([vR * cp - vp * sp, vR * sp + vp * cp, vz])
    bpos, rb, gb = hernquist_positions(nb, seed + 7919, Mb, bulge_a, rmax)
    ab = Md_a + Md_b
    rr, s2 = _jeans_sigma_r2_table(lambda x: _hernquist_rho(x, Mb, bulge_a),
                                   lambda x: _hernquist_mass(x, Mb, bulge_a) + Md * x ** 3 / (x * x + ab * ab) ** 1.5)
    sb = np.sqrt(_Interp(rr, s2)(rb))
    bvel = _spherical_gaussian_velocities(gb, bpos, rb, sb, sb)
    pos = np.concatenate([dpos, bpos], axis=1)
    vel = np.concatenate([dvel, bvel], axis=1)
    order = np.argsort((pos * pos).sum(0), kind="stable")
    return np.ascontiguousarray(pos[:, order]), np.ascontiguousarray(vel[:, order])


def log_shell_edges(nbins, rmin, rmax):
    """Squared edges r_k^2 of nbins log-spaced radial bins in [rmin, rmax]."""
    k = np.arange(nbins + 1, dtype=np.float64)
    r = rmin * (rmax / rmin) ** (k / nbins)
    return r * r


def uniform_edges(nbins, lo, hi):
    """nbins+1 uniform edges lo + k (hi-lo)/nbins (float64)."""
    k = np.arange(nbins + 1, dtype=np.float64)
    return lo + k * ((hi - lo) / nbins)


def error_model(Y, obs_sets, frac=0.02):
    """Observational errors: sigma_j = 2% of the target value for masses and
    v_los^2 moments; for Gauss-Hermite moments sigma_{p,n} = 2% of the
    aperture's h0 observable Y_{p,0} (an absolute 0.02 in h_n units).
    A target <= 0 masks the observable (sigma = 0)."""
    Y = np.asarray(Y, dtype=np.float64)
    sig = np.zeros_like(Y)
    off = 0
    for s in obs_sets:
        blk = Y[off:off + s.nobs].reshape(s.ncells, s.nmom)
        ref = blk[:, 0:1]
        sb = np.where(ref > 0, frac * ref, 0.0) * np.ones((1, s.nmom))
        sig[off:off + s.nobs] = sb.reshape(-1)
        off += s.nobs
    return sig


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
WORKLOADS = ("plain-fp64", "moving-priors", "flat-log", "sh-selfcons", "ifu-lut", "sh-tri", "sh-full")

_DEFAULT_N = {"plain-fp64": 20_000, "moving-priors": 1_000_000, "sh-selfcons": 8_000_000,
              "flat-log": 4_000_000, "ifu-lut": 4_000_000, "sh-tri": 4_000_000,
              "sh-full": 4_000_000}

# axis ratios of the triaxial workload (x : y : z)
TRI_AXES = (1.0, 0.8, 0.6)


# orientation and offset of the particle set of the workload with no symmetry
# (Euler angles z-y-z, radians; centre offset)
FULL_EULER = (0.5, 0.7, 0.3)
FULL_SHIFT = (0.05, -0.03, 0.02)


def rotated(pos, vel, euler=FULL_EULER, shift=FULL_SHIFT):
    """Positions rotated by the z-y-z Euler angles and shifted by `shift`,
    velocities rotated: a set with no mirror symmetry about the coordinate
    planes (every harmonic appears in its expansion)."""
    a, b, c = euler

    def rz(t):
        return np.array([[math.cos(t), -math.sin(t), 0.0], [math.sin(t), math.cos(t), 0.0], [0.0, 0.0, 1.0]])

    def ry(t):
        return np.array([[math.cos(t), 0.0, math.sin(t)], [0.0, 1.0, 0.0], [-math.sin(t), 0.0, math.cos(t)]])

    M = rz(a) @ ry(b) @ rz(c)
    return M @ pos + np.asarray(shift, np.float64)[:, None], M @ vel


def triaxial_hernquist(n, seed, axes=TRI_AXES):
    """A triaxial Hernquist-like particle set: an isotropic Hernquist
    realisation with positions and velocities stretched along the axes by
    `axes` (a synthetic triaxial mass distribution; not an equilibrium)."""
    pos, vel = hernquist_isotropic(n, seed)
    k = np.asarray(axes, np.float64)[:, None]
    return pos * k, vel * k


# --------------------------------------------------------------------------
# Aperture lookup tables (sky pixel -> aperture) for the 'lut' geometry
# --------------------------------------------------------------------------
def _pixel_centres(edges_x, edges_y):
    cx = 0.5 * (edges_x[:-1] + edges_x[1:])
    cy = 0.5 * (edges_y[:-1] + edges_y[1:])
    return np.meshgrid(cx, cy)          # (ny, nx) each


def voronoi_lut(edges_x, edges_y, generators, rmax=None):
    """Voronoi binning: each pixel belongs to the generator nearest to its
    centre (the lowest index on a tie); pixels whose centre lies beyond rmax
    from the origin (the instrument's footprint) belong to none (-1)."""
    X, Y = _pixel_centres(edges_x, edges_y)
    g = np.asarray(generators, np.float64)
    d2 = (X[..., None] - g[:, 0]) ** 2 + (Y[..., None] - g[:, 1]) ** 2
    lut = np.argmin(d2, axis=-1).astype(np.int32)
    if rmax is not None:
        lut[X * X + Y * Y >= rmax * rmax] = -1
    return lut


def slit_lut(edges_x, edges_y, pa_deg, width, u_edges, centre=(0.0, 0.0)):
    """A long slit at position angle pa_deg (from the X axis) through
    `centre`, `width` wide, cut into segments by u_edges along it: a pixel
    belongs to segment k if its centre, at (u, v) along / across the slit,
    has |v| < width/2 and u_edges[k] <= u < u_edges[k+1]; else to none."""
    X, Y = _pixel_centres(edges_x, edges_y)
    c, s = math.cos(math.radians(pa_deg)), math.sin(math.radians(pa_deg))
    dx, dy = X - centre[0], Y - centre[1]
    u = c * dx + s * dy
    v = -s * dx + c * dy
    k = np.searchsorted(u_edges, u, side="right") - 1
    ok = (np.abs(v) < 0.5 * width) & (k >= 0) & (k < len(u_edges) - 1)
    return np.where(ok, k, -1).astype(np.int32)


def gaussian_psf_table(sigma, bits=12):
    """A Gaussian PSF of dispersion sigma per sky axis as 2^bits quantiles,
    sigma * Phi^-1((k + 1/2) / 2^bits): a uniform 32-bit draw u picks entry
    u >> (32 - bits)."""
    from statistics import NormalDist
    nd = NormalDist()
    m = 1 << bits
    return sigma * np.array([nd.inv_cdf((k + 0.5) / m) for k in range(m)])


def ifu_generators(n, seed, rmax):
    """n Voronoi generators in the disc r < rmax, denser towards the centre
    (r = rmax u^0.7), as adaptive binning to a fixed signal-to-noise makes
    them."""
    g = rng(seed)
    r = rmax * g.random(n) ** 0.7
    phi = 2 * math.pi * g.random(n)
    return np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)


def _gh_set_annuli(nb, rmin, rmax, sigma_kernel, GM=1.0, a=1.0):
    e = log_shell_edges(nb, rmin, rmax)
    rmid = np.sqrt(np.sqrt(e[:-1] * e[1:]))
    S = np.sqrt(hernquist_sigma_iso(GM, a)(rmid))
    return ObservableSet("annulus", "gh", e, gh_V=np.zeros(nb), gh_S=S,
                         sigma_kernel=sigma_kernel)


def make_problem(name, n=None, precision=None, seed_model=None,
                 seed_target=None, with_target=True, nsteps=None, seeing=None):
    """Build the workload `name` (see module docstring), optionally at another
    particle count `n` with the same structure.  Weights and priors start at
    1/n.  eps is the workload's epsilon divided by the workload's nominal N
    (not by n): the relaxation rate of bin j, eps Y_j / sigma_j^2, then does
    not depend on how many particles a reduced test case uses."""
    nominal = _DEFAULT_N[name]
    if n is None:
        n = nominal
    if name == "plain-fp64":
        sm, st = seed_model or 1, seed_target or 2
        pos, vel = hernquist_isotropic(n, sm)
        tp = tv = None
        if with_target:
            tp, tv = hernquist_om_target(n, st, ra=1.0)
        ann = log_shell_edges(20, 0.05, 20.0)
        obs = [ObservableSet("shell", "mass", log_shell_edges(40, 0.05, 20.0)),
               ObservableSet("annulus", "mass", ann),
               ObservableSet("annulus", "vlos2", ann.copy())]
        pot = [PotentialComponent("hernquist", (1.0, 1.0))]
        prior = PriorSpec("flat")
        sin_i, cos_i = 0.0, 1.0
        prec = precision or "fp64"
        steps = nsteps or 2000
    elif name == "moving-priors":
        sm, st = seed_model or 3, seed_target or 4
        pos, vel = hernquist_isotropic(n, sm)
        tp = tv = None
        if with_target:
            tp, tv = hernquist_om_target(n, st, ra=1.0)
        obs = [ObservableSet("shell", "mass", log_shell_edges(100, 0.05, 20.0)),
               _gh_set_annuli(60, 0.05, 20.0, 0.1)]
        pot = [PotentialComponent("hernquist", (1.0, 1.0))]
        prior = PriorSpec("e_lc", nE=64, nL=32, period=25, hernquist=(1.0, 1.0))
        sin_i, cos_i = 0.0, 1.0
        prec = precision or "fp32c"
        steps = nsteps or 5000
    elif name == "flat-log":
        sm, st = seed_model or 5, seed_target or 6
        v0, Rc, q = 1.0, 0.1, 0.8
        pos, vel = log_flattened_realisation(n, sm, v0, Rc, q)
        tp = tv = None
        if with_target:
            tp, tv = log_flattened_realisation(n, st, v0, Rc, q, stream_frac=0.5)
        ap = uniform_edges(20, -2.0, 2.0)
        obs = [ObservableSet("grid", "mass", uniform_edges(64, -3.2, 3.2),
                             uniform_edges(64, -3.2, 3.2)),
               ObservableSet("grid", "gh", ap, ap.copy(),
                             gh_V=np.zeros(400), gh_S=np.full(400, v0 / math.sqrt(2.0)),
                             sigma_kernel=0.1)]
        pot = [PotentialComponent("log", (v0, Rc, q))]
        prior = PriorSpec("e_lz", nE=128, nL=64, period=25)
        inc = math.radians(60.0)
        sin_i, cos_i = math.sin(inc), math.cos(inc)
        prec = precision or "fp32c"
        steps = nsteps or 5000
    elif name == "ifu-lut":
        # the flat-log galaxy observed through a Voronoi-binned IFU and a
        # long slit (apertures of any shape by sky-pixel lookup tables)
        sm, st = seed_model or 5, seed_target or 6
        v0, Rc, q = 1.0, 0.1, 0.8
        pos, vel = log_flattened_realisation(n, sm, v0, Rc, q)
        tp = tv = None
        if with_target:
            tp, tv = log_flattened_realisation(n, st, v0, Rc, q, stream_frac=0.5)
        px = uniform_edges(160, -2.0, 2.0)
        vor = voronoi_lut(px, px, ifu_generators(300, 11, 2.0), rmax=2.0)
        sx = uniform_edges(256, -3.2, 3.2)
        slit = slit_lut(sx, sx, 30.0, 0.2, uniform_edges(40, -3.0, 3.0))
        S0 = v0 / math.sqrt(2.0)
        obs = [ObservableSet("grid", "mass", uniform_edges(64, -3.2, 3.2),
                             uniform_edges(64, -3.2, 3.2)),
               ObservableSet("lut", "gh", px, px.copy(), gh_V=np.zeros(300), gh_S=np.full(300, S0),
                             sigma_kernel=0.1, lut=vor, n_apertures=300),
               ObservableSet("lut", "gh", sx, sx.copy(), gh_V=np.zeros(40), gh_S=np.full(40, S0),
                             sigma_kernel=0.1, lut=slit, n_apertures=40)]
        if seeing:
            # the spectroscopic sets seen through a Gaussian PSF of
            # dispersion `seeing` per axis (one stream of draws per set)
            for k in (1, 2):
                obs[k] = replace(obs[k], psf_q=gaussian_psf_table(seeing), psf_seed=12345 + k)
        pot = [PotentialComponent("log", (v0, Rc, q))]
        prior = PriorSpec("e_lz", nE=128, nL=64, period=25)
        inc = math.radians(60.0)
        sin_i, cos_i = math.sin(inc), math.cos(inc)
        prec = precision or "fp32c"
        steps = nsteps or 5000
    elif name == "sh-tri":
        sm, st = seed_model or 12, seed_target or 13
        pos, vel = triaxial_hernquist(n, sm)
        tp = tv = None
        if with_target:
            tp, tv = triaxial_hernquist(n, st)
        e = log_shell_edges(60, 0.05, 20.0)
        rmid = np.sqrt(np.sqrt(e[:-1] * e[1:]))
        S = np.maximum(np.sqrt(hernquist_sigma_iso(1.0, 1.0)(rmid)), 0.05)
        obs = [ObservableSet("shell", "mass", log_shell_edges(100, 0.05, 20.0)),
               ObservableSet("annulus", "gh", e, gh_V=np.zeros(60), gh_S=S, sigma_kernel=0.1)]
        pot = [PotentialComponent("sh_tri", (256, 1e-3, 100.0, 50))]
        prior = PriorSpec("e_l2", 64, 32, 25)
        sin_i, cos_i = 0.0, 1.0
        prec = precision or "fp32c"
        steps = nsteps or 5000
    elif name == "sh-full":
        sm, st = seed_model or 14, seed_target or 15
        pos, vel = rotated(*triaxial_hernquist(n, sm))
        tp = tv = None
        if with_target:
            tp, tv = rotated(*triaxial_hernquist(n, st))
        e = log_shell_edges(60, 0.05, 20.0)
        rmid = np.sqrt(np.sqrt(e[:-1] * e[1:]))
        S = np.maximum(np.sqrt(hernquist_sigma_iso(1.0, 1.0)(rmid)), 0.05)
        obs = [ObservableSet("shell", "mass", log_shell_edges(100, 0.05, 20.0)),
               ObservableSet("annulus", "gh", e, gh_V=np.zeros(60), gh_S=S, sigma_kernel=0.1)]
        pot = [PotentialComponent("sh_full", (128, 1e-3, 100.0, 50))]
        prior = PriorSpec("e_l2", 64, 32, 25)
        sin_i, cos_i = 0.0, 1.0
        prec = precision or "fp32c"
        steps = nsteps or 5000
    elif name == "sh-selfcons":
        sm, st = seed_model or 9, seed_target or 10
        pos, vel = disc_bulge_realisation(n, sm)
        tp = tv = None
        if with_target:
            tp, tv = disc_bulge_realisation(n, st)
        e = log_shell_edges(60, 0.05, 20.0)
        rmid = np.sqrt(np.sqrt(e[:-1] * e[1:]))
        S = np.maximum(np.sqrt(hernquist_sigma_iso(0.75, 0.3)(rmid)), 0.05)
        obs = [ObservableSet("shell", "mass", log_shell_edges(100, 0.05, 20.0)),
               ObservableSet("annulus", "gh", e, gh_V=np.zeros(60), gh_S=S, sigma_kernel=0.1)]
        pot = [PotentialComponent("sh", (256, 1e-3, 100.0, 50))]
        prior = PriorSpec("flat")
        sin_i, cos_i = 0.0, 1.0
        prec = precision or "fp32c"
        steps = nsteps or 10000
    else:
        raise ValueError(f"unknown workload {name!r}")
    w0 = np.full(n, 1.0 / n)
    tw = None if tp is None else np.full(n, 1.0 / n)
    return Problem(name=name, n=n, pos=np.ascontiguousarray(pos),
                   vel=np.ascontiguousarray(vel), w0=w0, what0=w0.copy(),
                   potential=pot, obs=obs, incl_sin=sin_i, incl_cos=cos_i,
                   eps=0.05 / nominal, mu=1e-3, dt=0.01, alpha=0.02, prior=prior,
                   nsteps=steps, precision=prec, target_pos=tp, target_vel=tv,
                   target_w=tw)


# --------------------------------------------------------------------------
# Batched trial potentials: Hernquist stars in Hernquist + NFW potentials
# --------------------------------------------------------------------------
def nfw_rho_s(mass_ratio, r_s, M_star=1.0):
    """rho_s of an NFW halo whose mass inside 10 r_s is mass_ratio * M_star."""
    c = 10.0
    return mass_ratio * M_star / (4 * math.pi * r_s ** 3 * (math.log1p(c) - c / (1 + c)))


def _nfw_mass(r, rho_s, r_s):
    u = r / r_s
    return 4 * math.pi * rho_s * r_s ** 3 * (np.log1p(u) - u / (1 + u))


def hernquist_in_halo(n, seed, rho_s, r_s, ra=None, GM=1.0, a=1.0, rmax=100.0):
    """Hernquist tracer (positions by inverse CDF) with Gaussian velocities
    from the Jeans equation in the Hernquist + NFW potential (isotropic, or
    Osipkov-Merritt-like beta = r^2/(r^2 + ra^2))."""
    pos, r, g = hernquist_positions(n, seed, GM, a, rmax)
    rr, s2 = _jeans_sigma_r2_table(lambda x: _hernquist_rho(x, GM, a),
                                   lambda x: _hernquist_mass(x, GM, a) + _nfw_mass(x, rho_s, r_s), ra=ra)
    sr = np.sqrt(_Interp(rr, s2)(r))
    if ra is None:
        st = sr
    else:
        st = np.sqrt(1.0 - r * r / (r * r + ra * ra)) * sr
    vel = _spherical_gaussian_velocities(g, pos, r, sr, st)
    return pos, vel


HALO_MASS_RATIOS = (0.5, 1.0, 2.0, 4.0, 8.0, 16.0)
HALO_RS = tuple(float(v) for v in np.geomspace(1.0, 20.0, 8))


def make_scan(halos, true_halo, n=100_000, n_target=None, seed=21, precision="fp32c", target_ra=1.0):
    """One data set fitted in a sequence of trial potentials (Section 4):
    Hernquist stars (GM = a = 1) in Hernquist + NFW halos.  halos: list of
    (M_h/M_*, r_s/a) trial halos; true_halo: the halo of the target galaxy
    (Osipkov-Merritt-like anisotropy radius target_ra, None for isotropic;
    seed `seed`, n_target particles) whose observables every model fits.  Model m starts isotropic in its own trial
    potential (seed 1000 + m); all share the observables (100 shells + 60
    annuli x h0..h4 about the target's Jeans dispersion), flat priors and
    eps = 0.05 / n.  The targets are left to the caller to observe
    (Problem.target_* of every model hold the same galaxy)."""
    n_target = n_target or n
    rt, st = true_halo
    rho_t = nfw_rho_s(rt, st)
    tp, tv = hernquist_in_halo(n_target, seed, rho_t, st, ra=target_ra)
    tw = np.full(n_target, 1.0 / n_target)
    e = log_shell_edges(60, 0.05, 20.0)
    rmid = np.sqrt(np.sqrt(e[:-1] * e[1:]))
    rr, s2 = _jeans_sigma_r2_table(lambda x: _hernquist_rho(x),
                                   lambda x: _hernquist_mass(x) + _nfw_mass(x, rho_t, st))
    S = np.sqrt(_Interp(rr, s2)(rmid))
    obs = [ObservableSet("shell", "mass", log_shell_edges(100, 0.05, 20.0)),
           ObservableSet("annulus", "gh", e, gh_V=np.zeros(60), gh_S=S, sigma_kernel=0.1)]
    out = []
    for m, (ratio, r_s) in enumerate(halos):
        rho_s = nfw_rho_s(ratio, r_s)
        pos, vel = hernquist_in_halo(n, 1000 + m, rho_s, r_s)
        w0 = np.full(n, 1.0 / n)
        pot = [PotentialComponent("hernquist", (1.0, 1.0)), PotentialComponent("nfw", (rho_s, r_s))]
        out.append(Problem(name=f"scan-{m}", n=n, pos=np.ascontiguousarray(pos), vel=np.ascontiguousarray(vel),
                           w0=w0, what0=w0.copy(), potential=pot, obs=obs, incl_sin=0.0, incl_cos=1.0,
                           eps=0.05 / n, mu=1e-3, dt=0.01, alpha=0.02, prior=PriorSpec("flat"),
                           nsteps=1000, precision=precision, target_pos=tp, target_vel=tv, target_w=tw,
                           meta={"mass_ratio": ratio, "r_s": r_s, "rho_s": rho_s}))
    return out


def make_batch(nmodels=48, n_lo=100_000, n_hi=2_000_000, seed=7, n_scale=1.0, precision="fp32c",
               with_target=True):
    """The batched workload: model m uses halo (HALO_MASS_RATIOS[m // 8],
    HALO_RS[m % 8]) (the 6 x 8 grid for 48 models), N_m = floor(exp(U(ln
    n_lo, ln n_hi))) from one seeded stream (times n_scale for reduced
    tests), model seed 1000 + m and target seed 2000 + m (Osipkov-Merritt-
    like r_a = 1), observables as the moving-prior workload (100 shells +
    60 annuli x h0..h4), flat priors, eps = 0.05 / N_m (nominal N)."""
    g = rng(seed)
    Ns = np.floor(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), nmodels))).astype(np.int64)
    out = []
    for m in range(nmodels):
        ratio = HALO_MASS_RATIOS[(m // 8) % len(HALO_MASS_RATIOS)]
        r_s = HALO_RS[m % 8]
        rho_s = nfw_rho_s(ratio, r_s)
        n = max(1, int(Ns[m] * n_scale))
        pos, vel = hernquist_in_halo(n, 1000 + m, rho_s, r_s)
        tp = tv = tw = None
        if with_target:
            tp, tv = hernquist_in_halo(n, 2000 + m, rho_s, r_s, ra=1.0)
            tw = np.full(n, 1.0 / n)
        e = log_shell_edges(60, 0.05, 20.0)
        rmid = np.sqrt(np.sqrt(e[:-1] * e[1:]))
        rr, s2 = _jeans_sigma_r2_table(lambda x: _hernquist_rho(x), lambda x: _hernquist_mass(x) + _nfw_mass(x, rho_s, r_s))
        S = np.sqrt(_Interp(rr, s2)(rmid))
        obs = [ObservableSet("shell", "mass", log_shell_edges(100, 0.05, 20.0)),
               ObservableSet("annulus", "gh", e, gh_V=np.zeros(60), gh_S=S, sigma_kernel=0.1)]
        pot = [PotentialComponent("hernquist", (1.0, 1.0)), PotentialComponent("nfw", (rho_s, r_s))]
        w0 = np.full(n, 1.0 / n)
        out.append(Problem(name=f"batched-{m}", n=n, pos=np.ascontiguousarray(pos), vel=np.ascontiguousarray(vel),
                           w0=w0, what0=w0.copy(), potential=pot, obs=obs, incl_sin=0.0, incl_cos=1.0,
                           eps=0.05 / int(Ns[m]), mu=1e-3, dt=0.01, alpha=0.02, prior=PriorSpec("flat"),
                           nsteps=1000, precision=precision, target_pos=tp, target_vel=tv, target_w=tw,
                           meta={"mass_ratio": ratio, "r_s": r_s, "rho_s": rho_s, "N_nominal": int(Ns[m])}))
    return out
