"""The autotuner times real steps of the live model: every configuration it
tries yields the same FP32C state, so a tuned run equals an untuned run of
the same number of steps; a cached choice is applied without stepping."""
import numpy as np
import pytest

from oracle import m2m as O
from paper_1207_6403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402


def _problem(name, n):
    P = I.make_problem(name, n=n, precision="fp32c")
    Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
    return P.with_targets(Y)


@pytest.mark.parametrize("name", ["flat-log", "moving-priors"])
def test_autotune_advances_the_model_as_plain_steps_would(name, tmp_path):
    P = _problem(name, 30011)
    cache = str(tmp_path / "tune.jsonl")
    ctx = B.from_problem(P, "fp32c")
    tune = ctx.m2m_autotune(4, cache)
    assert tune["candidates"] >= 4 and not tune["from_cache"]
    assert tune["threads"] in (256, 512, 1024) and tune["pipeline"] & 6
    steps = ctx.m2m_steps_taken()
    assert steps == tune["candidates"] * 5
    ctx.m2m_step(7)
    g = ctx.state()
    y, _, _ = ctx.m2m_get_obs()
    ref = B.from_problem(P, "fp32c")
    ref.m2m_step(steps + 7)
    g0 = ref.state()
    y0, _, _ = ref.m2m_get_obs()
    for k in ("x", "y", "z", "vx", "vy", "vz", "w", "what"):
        assert np.array_equal(g[k], g0[k]), k
    assert np.array_equal(y, y0)
    # a second context of the same configuration takes the cached choice
    ctx2 = B.from_problem(P, "fp32c")
    t2 = ctx2.m2m_autotune(4, cache)
    assert t2["from_cache"] and t2["key"] == tune["key"]
    assert (t2["threads"], t2["pipeline"]) == (tune["threads"], tune["pipeline"])
    assert ctx2.m2m_steps_taken() == 0


def test_autotune_rejects_bad_arguments():
    P = _problem("plain-fp64", 2000)
    ctx = B.from_problem(P, "fp32c")
    with pytest.raises(B.M2MError):
        ctx.m2m_autotune(0)


def test_batch_autotune_keeps_models_equal_to_models_stepped_alone():
    problems = []
    for P in I.make_batch(nmodels=4, n_scale=0.004):
        Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
        problems.append(P.with_targets(Y))
    bt = B.m2m_batch_init("fp32c", problems)
    tune = bt.m2m_batch_autotune(3)
    assert tune["candidates"] == 3 and tune["choice"].startswith("pass blocks x")
    bt.m2m_batch_step(5)
    assert bt.m2m_batch_fused() == 2
    torch.cuda.synchronize()
    total = 3 * 2 * 3 + 5
    for m, P in enumerate(problems):
        g = bt.m2m_batch_context(m).state()
        alone = B.from_problem(P, "fp32c")
        alone.m2m_step(total)
        g0 = alone.state()
        for k in ("x", "y", "z", "vx", "vy", "vz", "w"):
            assert np.array_equal(g[k], g0[k]), (m, k)
        alone.m2m_free()
    bt.m2m_batch_free()
