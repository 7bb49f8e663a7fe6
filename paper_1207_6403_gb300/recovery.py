"""Recovery of the orbital anisotropy of a spherical target from different
initial particle models (Section 3 and its Fig. 1): the moving-prior
workload (Hernquist stars, Osipkov-Merritt-like target with r_a = 1, shells
and Gauss-Hermite annuli, (E, L^2/L_c^2) moving priors) started from an
isotropic, a radially and a tangentially anisotropic initial model, and
the anisotropy beta(r) of each weighted model measured by the library."""
import numpy as np

from . import inputs as I
from . import m2m as B

INITIAL = {
    "isotropic": lambda n, seed: I.hernquist_isotropic(n, seed),
    "radial": lambda n, seed: I.hernquist_om_target(n, seed, ra=0.3),
    "tangential": lambda n, seed: I.hernquist_const_beta(n, seed, -0.5),
}


def anisotropy(moments):
    """beta = 1 - (sigma_theta^2 + sigma_phi^2) / (2 sigma_r^2) per shell."""
    m = np.asarray(moments, np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        return 1.0 - (m[:, 2] + m[:, 3]) / (2.0 * m[:, 1])


def recovery(n, nsteps, r_edges, seed=3, precision="fp32c", device="cuda:0", initial=INITIAL,
             eps_scale=1.0):
    """Returns {name: (beta_initial, beta_final, record)} for every initial
    model, and the target's beta on the same shells (r_edges: edges of r).
    eps_scale multiplies the workload's adaptation rate epsilon."""
    P = I.make_problem("moving-priors", n=n, precision=precision)
    P.eps = P.eps * eps_scale
    Y = B.observe_targets(P, precision, device)
    P = P.with_targets(Y)
    e2 = np.asarray(r_edges, np.float64) ** 2
    out = {}
    for name, make in initial.items():
        pos, vel = make(n, seed)
        Q = I.Problem(**{**P.__dict__, "pos": pos, "vel": vel})
        ctx = B.from_problem(Q, precision, device=device)
        b0 = anisotropy(ctx.m2m_velocity_moments(e2))
        ctx.m2m_step(nsteps)
        b1 = anisotropy(ctx.m2m_velocity_moments(e2))
        out[name] = (b0, b1, ctx.m2m_get_record())
        ctx.m2m_free()
    tctx = B.m2m_init(precision, P.target_pos, P.target_vel, P.target_w, P.target_w, P.potential, P.obs,
                      B.params_of(P), None, None, None, device)
    target = anisotropy(tctx.m2m_velocity_moments(e2))
    tctx.m2m_free()
    return out, target
