"""The anisotropy analysis of the recovery experiment: velocity-ellipsoid
moments per spherical shell against the oracle (double sums in atomic
order: 1e-12 relative), after steps and with a pending weight update."""
import numpy as np
import pytest

from oracle import m2m as O
from paper_1207_6403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402
from paper_1207_6403_gb300 import recovery as RC  # noqa: E402


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_velocity_moments_match_the_oracle(prec):
    P = I.make_problem("moving-priors", n=30011, precision=prec)
    P = P.with_targets(O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos))
    ctx = B.from_problem(P, prec)
    ctx.m2m_set_lazy_update(True)
    ctx.m2m_step(7)                      # the last update pending: applied first
    e2 = I.log_shell_edges(12, 0.05, 20.0)
    m = ctx.m2m_velocity_moments(e2)
    g = ctx.state()
    ref = O.velocity_moments(g["x"], g["y"], g["z"], g["vx"], g["vy"], g["vz"], g["w"], e2)
    np.testing.assert_allclose(m, ref, rtol=1e-12, atol=1e-15 * np.abs(ref).max())
    np.testing.assert_allclose(RC.anisotropy(m), O.anisotropy(ref), rtol=1e-10)
    with pytest.raises(B.M2MError):
        ctx.m2m_velocity_moments(np.array([1.0, 0.5]))


def test_recovery_driver_runs_three_initial_models():
    out, target = RC.recovery(20011, 10, np.geomspace(0.2, 5.0, 5))
    assert set(out) == {"isotropic", "radial", "tangential"}
    for b0, b1, rec in out.values():
        assert b0.shape == b1.shape == (4,) and rec["step"] == 10
    assert out["radial"][0].mean() > 0.5 and out["tangential"][0].mean() < -0.3
    assert np.all(np.isfinite(target))
