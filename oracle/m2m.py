"""The M2M training step, written out plainly (oracle; test infrastructure only).

Section 2 of the paper: the weights w_i of an N-body model are adapted,
while its particles orbit in the potential, so that its observables match
those of a target galaxy: F = -1/2 chi^2 + mu S (Eq. 1) with
S = -sum_i w_i ln(w_i/w_hat_i) (Eq. 2) is maximised over the weights.
Section 2.1: flat priors w_hat_i = 1/N, or moving priors that follow the
weight distribution in integral-of-motion space.

One step t -> t+1, in this order:

1. push      KDK leapfrog: v += dt/2 a(x); x += dt v; v += dt/2 a(x) (a from
             analytic components and, optionally, a spherical-harmonic
             expansion of the particles themselves, see :mod:`oracle.sh`)
2. observe   y_j = sum_i w_i K_j(x_i, v_i) at the new positions, old weights
3. residual  Delta_j = (y_j - Y_j)/sigma_j (0 where sigma_j <= 0);
             Delta~_j <- alpha Delta_j + (1-alpha) Delta~_j;
             chi2 = sum_j Delta~_j^2, chi2_raw = sum_j Delta_j^2
4. update    G_i = mu (-ln(w_i/w_hat_i) - c) - sum_j K_ij Delta~_j/sigma_j,
             w_i <- w_i exp(eps dt G_i)   (c = 1: the derivative of Eq. 2)
5. priors    if moving and (t+1) % period == 0: w_hat_i = mean w over the
             cell of i, cells from (x_{t+1}, v_{t+1}), weights w_{t+1}
6. potential if it has a spherical-harmonic part and (t+1) % its period == 0:
             recompute its tables from (x_{t+1}, w_{t+1})
7. record    S_t, sum w_t (the weights that produced y), F_t = -chi2/2 + mu S_t

At initialisation Delta~ := Delta of an observe at (x_0, w_0).

Bin and cell membership is taken in the state precision (float64 or
float32) from values computed in a fixed order (see :func:`sky`,
:func:`cells_and_kernels`, :func:`prior_cells`) and compared with float64
edge tables: a value v is in cell j iff e_j <= v < e_{j+1}; anything else,
NaN included, is in no cell.
"""
from dataclasses import dataclass, field

import numpy as np

from . import gh as _gh
from . import philox as _philox
from . import sh as _sh
from . import sh_full as _shf
from .potentials import acceleration as _analytic_acceleration
from .potentials import potential as _analytic_potential


def state_dtype(precision):
    return np.float64 if precision == "fp64" else np.float32


# --------------------------------------------------------------------------
# potential: analytic components plus, optionally, a self-consistent
# spherical-harmonic component (kind 'sh', params (K, rmin, rmax, period),
# last in the list) whose tables are part of the state
# --------------------------------------------------------------------------
SH_KINDS = ("sh", "sh_tri", "sh_full")


def _split(comps):
    an = [c for c in comps if c.kind not in SH_KINDS]
    sh = [c for c in comps if c.kind in SH_KINDS]
    return an, (sh[0] if sh else None)


def sh_tables(x, y, z, w, comp):
    """(F, D, nodes) of the expansion of the weighted particles: the
    axisymmetric even-l expansion (kind 'sh', :mod:`oracle.sh`), the
    triaxial one (kind 'sh_tri': even l, even m >= 0, l <= 8) or the general
    one (kind 'sh_full': every l <= 4 and m, :mod:`oracle.sh_full`)."""
    K, rmin, rmax = int(comp.params[0]), comp.params[1], comp.params[2]
    rn = _sh.nodes(rmin, rmax, K)
    if comp.kind == "sh_tri":
        return _shf.tri_tables(x, y, z, w, rn)
    if comp.kind == "sh_full":
        return _shf.full_tables(x, y, z, w, rn)
    A, B = _sh.coefficients(x, y, z, w, rn)
    F, D = _sh.tables(A, B, rn)
    return F, D, rn


def acceleration(x, y, z, comps, sh=None):
    """Analytic components in order, then the expansion (float64, rounded
    to the state precision) if the potential has one."""
    ax, ay, az = _analytic_acceleration(x, y, z, _split(comps)[0])
    if sh is not None:
        T = x.dtype.type
        kind = _split(comps)[1].kind
        if kind == "sh_tri":
            bx, by, bz = _shf.tri_acceleration(x, y, z, *sh)
        elif kind == "sh_full":
            bx, by, bz = _shf.full_acceleration(x, y, z, *sh)
        else:
            bx, by, bz = _sh.acceleration(x, y, z, *sh)
        ax, ay, az = ax + bx.astype(T), ay + by.astype(T), az + bz.astype(T)
    return ax, ay, az


def potential(x, y, z, comps, sh=None):
    phi = _analytic_potential(x, y, z, _split(comps)[0])
    if sh is not None:
        kind = _split(comps)[1].kind
        if kind == "sh_tri":
            phi = phi + _shf.tri_potential(x, y, z, *sh).astype(x.dtype)
        elif kind == "sh_full":
            phi = phi + _shf.full_potential(x, y, z, *sh).astype(x.dtype)
        else:
            phi = phi + _sh.potential(x, y, z, *sh).astype(x.dtype)
    return phi


# --------------------------------------------------------------------------
# 1. push
# --------------------------------------------------------------------------
def kdk(x, y, z, vx, vy, vz, comps, dt, sh=None):
    """One kick-drift-kick step in the dtype of the arrays; returns new arrays.

    dt/2 and dt are rounded once from float64 to the state precision."""
    T = x.dtype.type
    h = T(np.float64(0.5) * np.float64(dt))
    d = T(dt)
    ax, ay, az = acceleration(x, y, z, comps, sh)
    vx = vx + h * ax
    vy = vy + h * ay
    vz = vz + h * az
    x = x + d * vx
    y = y + d * vy
    z = z + d * vz
    ax, ay, az = acceleration(x, y, z, comps, sh)
    vx = vx + h * ax
    vy = vy + h * ay
    vz = vz + h * az
    return x, y, z, vx, vy, vz


# --------------------------------------------------------------------------
# 2. observables
# --------------------------------------------------------------------------
def bin_index(v, edges):
    """Cell j with edges[j] <= v < edges[j+1] (compared in float64), else -1."""
    e = np.asarray(edges, dtype=np.float64)
    vd = np.asarray(v).astype(np.float64)
    j = np.searchsorted(e, vd, side="right") - 1
    bad = (j < 0) | (j >= len(e) - 1) | np.isnan(vd)
    return np.where(bad, -1, j).astype(np.int64)


def sky(x, y, z, vx, vy, vz, sin_i, cos_i):
    """Sky-plane coordinates and line-of-sight velocity for the line of sight
    s = (0, sin i, cos i), in the state precision:
    X = x, Y = z*sin i - y*cos i, v_los = vy*sin i + vz*cos i."""
    T = x.dtype.type
    s, c = T(sin_i), T(cos_i)
    return x, z * s - y * c, vy * s + vz * c


def seeing(X, Ys, s, k, epoch):
    """The sky position of each particle as seen through the set's PSF
    (seeing): displaced by (q[u0 >> (32 - b)], q[u1 >> (32 - b)]), q the
    set's table of 2^b displacement quantiles along one axis (rounded to the
    state precision), (u0, u1) the first two words of Philox4x32-10 at
    counter (i, epoch mod 2^32, k, epoch >> 32) and key (psf_seed, 0), i the
    particle index, k the set's index and epoch the number of pushes the
    positions have had; the sum is taken in the state precision."""
    T = X.dtype.type
    q = np.asarray(s.psf_q, dtype=np.float64).astype(T)
    b = int(round(np.log2(q.size)))
    i = np.arange(X.shape[0], dtype=np.uint64)
    e = int(epoch)
    u = _philox.philox4x32_10(i, e & 0xFFFFFFFF, k, e >> 32, s.psf_seed, 0)
    sh = np.uint32(32 - b)
    return X + q[u[0] >> sh], Ys + q[u[1] >> sh]


def cells_and_kernels(x, y, z, vx, vy, vz, obs_sets, sin_i, cos_i, epoch=0):
    """Per observable set: (cell index per particle, K per particle (n, nmom)).
    epoch: the number of pushes the positions have had (draws of the sets
    with a PSF)."""
    X0, Ys0, _ = sky(x, y, z, vx, vy, vz, sin_i, cos_i)
    # the kernel values are float64 functions of the stored state
    vd = (np.asarray(vy, np.float64) * np.float64(sin_i)
          + np.asarray(vz, np.float64) * np.float64(cos_i))
    out = []
    for k, s in enumerate(obs_sets):
        X, Ys = (X0, Ys0) if getattr(s, "psf_q", None) is None else seeing(X0, Ys0, s, k, epoch)
        if s.geom == "shell":
            cell = bin_index((x * x + y * y) + z * z, s.edges_x)
        elif s.geom == "annulus":
            cell = bin_index(X * X + Ys * Ys, s.edges_x)
        elif s.geom == "grid":
            ix = bin_index(X, s.edges_x)
            iy = bin_index(Ys, s.edges_y)
            cell = np.where((ix >= 0) & (iy >= 0), iy * s.nx + ix, -1)
        elif s.geom == "lut":
            # the sky pixel as for a grid, then the aperture that owns it
            ix = bin_index(X, s.edges_x)
            iy = bin_index(Ys, s.edges_y)
            inside = (ix >= 0) & (iy >= 0)
            lut = np.asarray(s.lut, np.int64).reshape(s.ny, s.nx)
            cell = np.where(inside, lut[np.where(inside, iy, 0), np.where(inside, ix, 0)], -1)
        else:
            raise ValueError(s.geom)
        if s.quant == "mass":
            K = np.ones((x.shape[0], 1))
        elif s.quant == "vlos2":
            K = (vd * vd)[:, None]
        elif s.quant == "gh":
            cc = np.where(cell >= 0, cell, 0)
            V = np.asarray(s.gh_V, np.float64)[cc]
            S = np.asarray(s.gh_S, np.float64)[cc]
            K = _gh.gh_kernel((vd - V) / S, s.sigma_kernel / S)
        else:
            raise ValueError(s.quant)
        out.append((cell, K))
    return out


def observe_from(kern, w, obs_sets):
    """y = concatenation over sets of sum_i w_i K_i into each cell (cell-major,
    moment-minor), summed in float64."""
    ys = []
    for (cell, K), s in zip(kern, obs_sets):
        m = cell >= 0
        blk = np.zeros((s.ncells, s.nmom))
        for n in range(s.nmom):
            blk[:, n] = np.bincount(cell[m], weights=w[m] * K[m, n],
                                    minlength=s.ncells)
        ys.append(blk.reshape(-1))
    return np.concatenate(ys)


def observe(x, y, z, vx, vy, vz, w, obs_sets, sin_i, cos_i, epoch=0):
    kern = cells_and_kernels(x, y, z, vx, vy, vz, obs_sets, sin_i, cos_i, epoch)
    return observe_from(kern, np.asarray(w, np.float64), obs_sets)


def velocity_moments(x, y, z, vx, vy, vz, w, r2_edges):
    """Velocity-ellipsoid moments per spherical shell (edges of r^2,
    membership as for shell sets): columns sum w, sum w v_r^2,
    sum w v_theta^2, sum w v_phi^2, the velocities float64 functions of the
    stored state: v_r = x.v / r, v_phi = (x vy - y vx) / R, v_theta^2 =
    v^2 - v_r^2 - v_phi^2 (v_r = 0 at r = 0, v_phi = 0 at R = 0)."""
    cell = bin_index((x * x + y * y) + z * z, r2_edges)
    X, Y, Z, U, V, W = (np.asarray(a, np.float64) for a in (x, y, z, vx, vy, vz))
    r = np.sqrt(X * X + Y * Y + Z * Z)
    R = np.sqrt(X * X + Y * Y)
    vr = np.where(r > 0, (X * U + Y * V + Z * W) / np.where(r > 0, r, 1.0), 0.0)
    vp = np.where(R > 0, (X * V - Y * U) / np.where(R > 0, R, 1.0), 0.0)
    v2 = U * U + V * V + W * W
    vt2 = v2 - vr * vr - vp * vp
    m = cell >= 0
    nsh = len(r2_edges) - 1
    out = np.zeros((nsh, 4))
    for k, q in enumerate((np.ones_like(r), vr * vr, vt2, vp * vp)):
        out[:, k] = np.bincount(cell[m], weights=np.asarray(w, np.float64)[m] * q[m], minlength=nsh)
    return out


def anisotropy(moments):
    """beta = 1 - (sigma_theta^2 + sigma_phi^2) / (2 sigma_r^2) per shell
    (no mean streaming assumed), NaN where a shell is empty."""
    m = np.asarray(moments, np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        return 1.0 - (m[:, 2] + m[:, 3]) / (2.0 * m[:, 1])


# --------------------------------------------------------------------------
# 3. residuals
# --------------------------------------------------------------------------
def residual(yv, Y, sigma, Dt_prev, alpha, first):
    """Returns (Delta, Delta~, coef = Delta~/sigma, chi2, chi2_raw)."""
    valid = sigma > 0
    ss = np.where(valid, sigma, 1.0)
    Delta = np.where(valid, (yv - Y) / ss, 0.0)
    if first:
        Dt = Delta.copy()
    else:
        Dt = alpha * Delta + (1.0 - alpha) * Dt_prev
    coef = np.where(valid, Dt / ss, 0.0)
    return Delta, Dt, coef, float(np.sum(Dt * Dt)), float(np.sum(Delta * Delta))


# --------------------------------------------------------------------------
# 4. weight update, entropy, merit
# --------------------------------------------------------------------------
def kernel_dot(kern, coef, obs_sets, n):
    """sum_j K_ij coef_j per particle (sets in order, moments in order)."""
    dot = np.zeros(n)
    off = 0
    for (cell, K), s in zip(kern, obs_sets):
        m = cell >= 0
        for k in range(s.nmom):
            dot[m] += K[m, k] * coef[off + cell[m] * s.nmom + k]
        off += s.nobs
    return dot


def entropy(w, what):
    """S = -sum_i w_i ln(w_i/w_hat_i) (Eq. 2), terms with w_i = 0 are 0."""
    m = w > 0
    return float(-np.sum(w[m] * np.log(w[m] / what[m])))


def update_weights(w, what, dot, eps, mu, dt, entropy_const=1.0):
    """w_i <- w_i exp(eps dt G_i), G_i = mu(-ln(w_i/w_hat_i) - c) - dot_i."""
    w_new = w.copy()
    m = w > 0
    G = mu * (-np.log(w[m] / what[m]) - entropy_const) - dot[m]
    w_new[m] = w[m] * np.exp(eps * dt * G)
    return w_new


def merit(chi2, S, mu):
    """F = -1/2 chi^2 + mu S (Eq. 1)."""
    return -0.5 * chi2 + mu * S


# --------------------------------------------------------------------------
# 5. priors
# --------------------------------------------------------------------------
def _count_edges_le(v, lo, hi, ncell):
    """Number of interior edges e_k = lo + k*((hi-lo)/ncell), k = 1..ncell-1,
    with e_k <= v (float64 compare); NaN counts 0.  Result in [0, ncell-1]."""
    width = (np.float64(hi) - np.float64(lo)) / np.float64(ncell)
    k = np.arange(1, ncell, dtype=np.float64)
    e = np.float64(lo) + k * width
    vd = np.asarray(v).astype(np.float64)
    cnt = np.searchsorted(e, vd, side="right")
    return np.where(np.isnan(vd), 0, cnt).astype(np.int64)


def prior_cells(x, y, z, vx, vy, vz, prior, comps, sh=None):
    """Cell of every particle in integral-of-motion space (Section 2.1).

    Computed in the state precision, in this order:
      v2 = (vx*vx + vy*vy) + vz*vz;  E = 0.5*v2 + Phi(x)
      'e_lz': Lz = x*vy - y*vx; cells on [min E, max E] x [-max|Lz|, max|Lz|]
      'e_l2': L = x cross v, L2 = (Lx*Lx + Ly*Ly) + Lz*Lz; cells on
              [min E, max E] x [0, max L2] (for potentials without a
              symmetry axis, where L_z is not conserved: E is, and L^2 is
              approximately conserved while the potential is nearly round;
              Section 2.1's cells of approximately conserved quantities)
      'e_lc': L = x cross v, L2 = (Lx*Lx + Ly*Ly) + Lz*Lz; for the Hernquist
              (GM, a) circular orbit of energy E (E < 0):
                ed = E*k (k = a/GM), sq = sqrt(1 - 8*ed),
                s = (-1 - sq)/(4*ed)   [= (r_c + a)/a],
                sm = s - 1, Lc2 = gma*(((sm*sm)*sm)/(s*s))   (gma = GM*a),
                X = L2/Lc2;
              cells on [min E, 0) x [0, 1]; E >= 0 -> the extra cell nE*nL.
    Returns int64 cell ids.
    """
    T = x.dtype.type
    v2 = (vx * vx + vy * vy) + vz * vz
    with np.errstate(divide="ignore", invalid="ignore"):
        E = T(0.5) * v2 + potential(x, y, z, comps, sh)
        if prior.kind == "e_lz":
            Lz = x * vy - y * vx
            lo, hi = np.float64(E.min()), np.float64(E.max())
            Lm = np.float64(np.abs(Lz).max())
            iE = _count_edges_le(E, lo, hi, prior.nE)
            iL = _count_edges_le(Lz, -Lm, Lm, prior.nL)
            return iE * prior.nL + iL
        if prior.kind == "e_l2":
            Lx = y * vz - z * vy
            Ly = z * vx - x * vz
            Lz = x * vy - y * vx
            L2 = (Lx * Lx + Ly * Ly) + Lz * Lz
            lo, hi = np.float64(E.min()), np.float64(E.max())
            iE = _count_edges_le(E, lo, hi, prior.nE)
            iL = _count_edges_le(L2, 0.0, np.float64(L2.max()), prior.nL)
            return iE * prior.nL + iL
        if prior.kind == "e_lc":
            GM, a = prior.hernquist
            k = T(a / GM)
            gma = T(GM * a)
            Lx = y * vz - z * vy
            Ly = z * vx - x * vz
            Lz = x * vy - y * vx
            L2 = (Lx * Lx + Ly * Ly) + Lz * Lz
            ed = E * k
            sq = np.sqrt(T(1) - T(8) * ed)
            s = (T(-1) - sq) / (T(4) * ed)
            sm = s - T(1)
            Lc2 = gma * (((sm * sm) * sm) / (s * s))
            X = L2 / Lc2
            lo = np.float64(E.min())
            iE = _count_edges_le(E, lo, 0.0, prior.nE)
            iL = _count_edges_le(X, 0.0, 1.0, prior.nL)
            cell = iE * prior.nL + iL
            return np.where(E >= 0, prior.nE * prior.nL, cell).astype(np.int64)
    raise ValueError(prior.kind)


def prior_means(w, cells, ncells):
    """w_hat_i = (sum of w over i's cell) / (number of particles in it)."""
    sums = np.bincount(cells, weights=w, minlength=ncells)
    cnt = np.bincount(cells, minlength=ncells)
    return sums[cells] / cnt[cells]


# --------------------------------------------------------------------------
# 6. the step loop
# --------------------------------------------------------------------------
@dataclass
class State:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    w: np.ndarray
    what: np.ndarray
    Dt: np.ndarray
    coef: np.ndarray
    t: int = 0
    y_obs: np.ndarray = None
    Delta: np.ndarray = None
    history: list = field(default_factory=list)
    sh: tuple = None
    epoch: int = 0               # pushes the positions have had

    @property
    def pos(self):
        return (self.x, self.y, self.z)

    @property
    def vel(self):
        return (self.vx, self.vy, self.vz)


def init(problem, precision=None):
    """State at t = 0: positions in the state precision, w = w0, w_hat =
    what0, Delta~ = Delta of the initial observe."""
    T = state_dtype(precision or problem.precision)
    x, y, z = (np.ascontiguousarray(a, dtype=T) for a in problem.pos)
    vx, vy, vz = (np.ascontiguousarray(a, dtype=T) for a in problem.vel)
    w = np.array(problem.w0, dtype=np.float64)
    what = np.array(problem.what0, dtype=np.float64)
    yv = observe(x, y, z, vx, vy, vz, w, problem.obs, problem.incl_sin,
                 problem.incl_cos)
    Delta, Dt, coef, _, _ = residual(yv, problem.Y, problem.sigma, None,
                                     problem.alpha, True)
    st = State(x, y, z, vx, vy, vz, w, what, Dt, coef, 0, yv, Delta)
    shc = _split(problem.potential)[1]
    if shc is not None:
        st.sh = sh_tables(x, y, z, w, shc)
    return st


def step(st, problem, push=True):
    """Advance `st` by one M2M step in place; returns the step's record."""
    P = problem
    w_used = st.w
    S_t = entropy(st.w, st.what)
    sumw_t = float(np.sum(st.w))
    if push:
        st.x, st.y, st.z, st.vx, st.vy, st.vz = kdk(
            st.x, st.y, st.z, st.vx, st.vy, st.vz, P.potential, P.dt, st.sh)
        st.epoch += 1
    kern = cells_and_kernels(st.x, st.y, st.z, st.vx, st.vy, st.vz, P.obs,
                             P.incl_sin, P.incl_cos, st.epoch)
    yv = observe_from(kern, w_used, P.obs)
    Delta, Dt, coef, chi2, chi2_raw = residual(yv, P.Y, P.sigma, st.Dt,
                                               P.alpha, False)
    dot = kernel_dot(kern, coef, P.obs, st.w.shape[0])
    st.w = update_weights(st.w, st.what, dot, P.eps, P.mu, P.dt,
                          P.entropy_const)
    st.t += 1
    if P.prior.kind != "flat" and st.t % P.prior.period == 0:
        cells = prior_cells(st.x, st.y, st.z, st.vx, st.vy, st.vz, P.prior,
                            P.potential, st.sh)
        st.what = prior_means(st.w, cells, P.prior.ncells)
    shc = _split(P.potential)[1]
    if shc is not None and st.t % int(shc.params[3]) == 0:
        st.sh = sh_tables(st.x, st.y, st.z, st.w, shc)
    st.Dt, st.coef, st.y_obs, st.Delta = Dt, coef, yv, Delta
    rec = dict(t=st.t, chi2=chi2, chi2_raw=chi2_raw, S=S_t, sum_w=sumw_t,
               F=merit(chi2, S_t, P.mu))
    st.history.append(rec)
    return rec


def run(problem, nsteps, precision=None, push=True, state=None):
    """Initialise (unless `state` is given) and take `nsteps` steps."""
    st = state if state is not None else init(problem, precision)
    for _ in range(nsteps):
        step(st, problem, push=push)
    return st
