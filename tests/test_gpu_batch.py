"""Batched trial potentials: many independent models advanced together.

A batch must give, model by model, exactly what stepping that model alone
through its own context gives (same kernels; the observable sums are exact
integers, so the number of blocks a model gets does not change them), and
one model is checked against the oracle.
"""
import numpy as np
import pytest

from oracle import m2m as O
from paper_1207_6403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402


def _with_targets(P):
    Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
    return P.with_targets(Y)


def _batch_problems(nmodels=5, n_scale=0.004):
    return [_with_targets(P) for P in I.make_batch(nmodels=nmodels, n_scale=n_scale)]


def _alone(P, nsteps):
    ctx = B.from_problem(P, "fp32c")
    ctx.m2m_step(nsteps)
    g = ctx.state()
    y, _, _ = ctx.m2m_get_obs()
    h = ctx.m2m_get_history(1, nsteps)
    ctx.m2m_free()
    return g, y, h


def _compare(bt, problems, nsteps, alone_steps=None):
    for m, P in enumerate(problems):
        ctx = bt.m2m_batch_context(m)
        g = ctx.state()
        y, _, _ = ctx.m2m_get_obs()
        h = ctx.m2m_get_history(1, nsteps)
        g1, y1, h1 = _alone(P, alone_steps or nsteps)
        for k in ("x", "y", "z", "vx", "vy", "vz", "w", "what"):
            assert np.array_equal(g[k], g1[k]), (m, k)
        assert np.array_equal(y, y1), m
        # S and sum w are accumulated per thread in float before the double
        # block sums, so they depend on how particles are grouped into blocks
        # (~1e-8 relative); chi^2 is a double sum of the same terms (exact
        # observables), grouped by observable slices that differ between the
        # fused batch and a persistent launch: equal to rounding
        for a, b in zip(h, h1):
            assert a["step"] == b["step"]
            assert a["chi2"] == pytest.approx(b["chi2"], rel=1e-13)
            assert a["sum_w"] == pytest.approx(b["sum_w"], rel=1e-6)
            assert a["S"] == pytest.approx(b["S"], rel=1e-5, abs=1e-6)


def test_batch_equals_models_stepped_alone_with_graph_replay():
    problems = _batch_problems()
    bt = B.m2m_batch_init("fp32c", problems)
    bt.m2m_batch_step(30)
    assert bt.m2m_batch_fused() == 2          # one launch per stage, captured in a graph
    bt.m2m_batch_step(30)                      # replays the captured graph
    assert bt.m2m_batch_fused() == 2
    torch.cuda.synchronize()
    _compare(bt, problems, 60)
    bt.m2m_batch_free()


def test_batch_with_moving_priors():
    problems = []
    for k in range(3):
        P = I.make_problem("moving-priors", n=3000 + 1700 * k, seed_model=40 + k, seed_target=50 + k)
        P.prior = I.PriorSpec("e_lc", 8, 4, 10, (1.0, 1.0))
        problems.append(_with_targets(P))
    bt = B.m2m_batch_init("fp32c", problems)
    bt.m2m_batch_step(25)
    assert bt.m2m_batch_fused() == 2
    torch.cuda.synchronize()
    _compare(bt, problems, 25)
    bt.m2m_batch_free()


def test_batch_of_different_layouts_falls_back_to_one_by_one():
    problems = [_with_targets(I.make_problem("plain-fp64", n=2000, precision="fp32c")),
                _with_targets(I.make_problem("moving-priors", n=3000))]
    problems[1].prior = I.PriorSpec("flat")
    bt = B.m2m_batch_init("fp32c", problems)
    bt.m2m_batch_step(12)
    assert bt.m2m_batch_fused() == 0
    torch.cuda.synchronize()
    _compare(bt, problems, 12)
    bt.m2m_batch_free()


@pytest.mark.parametrize("model", [0, 2])
def test_batch_model_weights_and_observables_on_the_gpu_orbits(model):
    """A model of a fused batch (Hernquist + NFW halo; the NFW force is float
    on the GPU and float64 rounded to float in the oracle, so the orbits part
    by rounding): every step the oracle takes that model's new positions
    from the GPU and does the scatter, residual and weight update itself;
    after 300 steps every weight agrees to 1e-4 relative and every
    observable to 1e-5 of its scale, no particle left out."""
    problems = _batch_problems(nmodels=3, n_scale=0.01)
    bt = B.m2m_batch_init("fp32c", problems)
    P = problems[model]
    st = O.init(P, "fp32c")
    for _ in range(300):
        bt.m2m_batch_step(1)
        g = bt.m2m_batch_context(model).state()
        st.x, st.y, st.z, st.vx, st.vy, st.vz = (g[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz"))
        O.step(st, P, push=False)
    assert bt.m2m_batch_fused() >= 1
    ctx = bt.m2m_batch_context(model)
    g = ctx.state()
    y, _, _ = ctx.m2m_get_obs()
    np.testing.assert_allclose(g["w"], st.w, rtol=1e-4)
    scale = np.maximum(np.maximum(np.abs(st.y_obs), P.sigma / 0.02), 1e-300)
    err = np.abs(y - st.y_obs) / scale
    assert err.max() <= 1e-5, (err.max(), err.argmax())
    bt.m2m_batch_free()


def test_batch_model_against_oracle():
    problems = _batch_problems(nmodels=3)
    bt = B.m2m_batch_init("fp32c", problems)
    bt.m2m_batch_step(40)
    torch.cuda.synchronize()
    P = problems[2]
    ctx = bt.m2m_batch_context(2)
    g = ctx.state()
    y, _, _ = ctx.m2m_get_obs()
    st = O.run(P, 40, precision="fp32c")
    # NFW force: float32 evaluation vs float64 rounded to float32 (the
    # weights and observables are checked on the GPU's own orbits above)
    for k in ("x", "y", "z"):
        np.testing.assert_allclose(g[k], getattr(st, k), rtol=0, atol=2e-5 * np.abs(getattr(st, k)).max())
    bt.m2m_batch_free()
