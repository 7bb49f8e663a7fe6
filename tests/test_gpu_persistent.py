"""Persistent multi-step launches (one cooperative launch per run of steps
up to a prior recompute, the residual between two grid barriers) against
the same steps taken as one pass launch and one residual launch each:
positions, velocities, weights, priors, observables, Delta and Delta~
bit-identical (the same per-particle and per-observable arithmetic, exact
integer histogram sums), also with heavy particles whose histogram terms
take the high-part path.  The records are sums over other partitions of
the same terms (the persistent blocks hold contiguous particle ranges and
observable slices): chi^2 (double terms) equal to 1e-12 relative; S and
sum w, whose per-thread partials are float sums of other particles, to
1e-6 of sum w (the FP32C records' stated accuracy).  And the
bounded grid-barrier wait: a launch whose block 0 never arrives records
M2M_ERR_TIMEOUT within the wait limit, and the GPU stays usable."""
import time
from dataclasses import replace

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


def _heavy(P, frac=0.005, factor=200.0):
    """A few particles at `factor` times their weight: their histogram terms
    exceed 2^31 fixed-point units, the path that carries a high part."""
    w0 = P.w0.copy()
    idx = np.random.default_rng(7).choice(P.n, size=max(1, int(frac * P.n)), replace=False)
    w0[idx] *= factor
    return replace(P, w0=w0)


@pytest.mark.parametrize("name,n,heavy", [("flat-log", 40_013, False), ("moving-priors", 30_011, False),
                                          ("ifu-lut", 20_021, False), ("flat-log", 3_000_017, False),
                                          ("flat-log", 50_021, True), ("ifu-lut", 30_011, True)])
def test_persistent_launches_equal_separate_launches(name, n, heavy):
    """Separate launches against persistent launches."""
    P = _problem(name, n)
    if heavy:
        P = _heavy(P)
    out = []
    for persist in (False, True):
        ctx = B.from_problem(P, "fp32c")
        ctx.m2m_set_persistent(persist)
        ctx.m2m_set_timing(True)
        ctx.m2m_step(7)           # a call shorter than the prior period
        ctx.m2m_step(55)          # crosses the recomputes at steps 25 and 50
        tm = ctx.m2m_get_timing()
        y, D, Dt = ctx.m2m_get_obs()
        hist = ctx.m2m_get_history(1, 62)
        out.append((ctx.state(), y, D, Dt, hist, tm))
        ctx.m2m_free()
    g0, y0, D0, d0, h0, t0 = out[0]
    assert t0["launches"]["steps"] == 0
    for g1, y1, D1, d1, h1, t1 in out[1:]:
        assert t1["launches"]["steps"] >= 3 and t1["steps"]["steps"] == 62
        for k in g0:
            assert np.array_equal(g0[k], g1[k]), k
        assert np.array_equal(y0, y1) and np.array_equal(D0, D1) and np.array_equal(d0, d1)
        for r0, r1 in zip(h0, h1):
            assert r0["step"] == r1["step"]
            for k in ("chi2", "chi2_raw", "max_abs_dt"):
                assert r1[k] == pytest.approx(r0[k], rel=1e-12), k
            for k in ("S", "sum_w"):
                assert abs(r1[k] - r0[k]) <= 1e-6 * abs(r0["sum_w"]), k
            assert r1["F"] == pytest.approx(r0["F"], rel=1e-12, abs=1e-8)


def test_persistent_lazy_single_steps_equal_one_call():
    """One step per call with lazy updates (the e2e loop) equals one call of
    all the steps, both persistent."""
    P = _problem("flat-log", 25_013)
    a = B.from_problem(P, "fp32c")
    a.m2m_step(30)
    ga = a.state()
    b = B.from_problem(P, "fp32c")
    b.m2m_set_lazy_update(True)
    for _ in range(30):
        b.m2m_step(1)
    gb = b.state()
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    a.m2m_free()
    b.m2m_free()


def test_grid_barrier_wait_runs_out_and_reports_timeout():
    P = _problem("flat-log", 200_003)
    ctx = B.from_problem(P, "fp32c")
    ctx.m2m_step(2)
    ctx.m2m_get_record()
    ctx.m2m_test_barrier_stall(20_000_000)          # 20 ms per wait
    t0 = time.perf_counter()
    ctx.m2m_step(1)
    with pytest.raises(B.M2MError) as e:
        ctx.m2m_get_record()
    assert e.value.code == -4 and "wait" in str(e.value)
    assert time.perf_counter() - t0 < 5.0
    ctx.m2m_free()
    # the GPU and a new context are unaffected
    c2 = B.from_problem(P, "fp32c")
    c2.m2m_step(3)
    assert np.isfinite(c2.m2m_get_record()["chi2"])
    c2.m2m_free()
