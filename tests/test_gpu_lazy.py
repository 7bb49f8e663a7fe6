"""Lazy weight updates: a model stepped one call per step with the update
of each call's last step left pending (and fused into the next call's
pass) has the same records, observables and state as one whose calls each
end with an update-only pass; every call that reads or changes the state
applies a pending update first.  Tolerances: positions, weights,
observables, chi^2 bit-identical in FP32C (FP64 histograms are double
atomic sums: 1e-10 relative); FP32C: sum w of the records to 1e-6
relative, the entropy S to 2e-6 sum w (its float logarithms are taken of
other arguments by the fused pass)."""
import numpy as np
import pytest

from oracle import m2m as O
from paper_1207_6403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402

KEYS = ("x", "y", "z", "vx", "vy", "vz", "w", "what")


def _problem(name, n, prec):
    P = I.make_problem(name, n=n, precision=prec)
    Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
    return P.with_targets(Y)


def _raw(ctx):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in ctx.t.items()}


@pytest.mark.parametrize("name,prec", [("moving-priors", "fp32c"), ("flat-log", "fp32c"),
                                       ("moving-priors", "fp64")])
def test_one_step_per_call_with_host_io_matches_immediate_updates(name, prec):
    """30 calls of m2m_set_targets + m2m_step(1) + m2m_get_record (a prior
    recompute at step 25 included)."""
    P = _problem(name, 20011, prec)
    rng = np.random.default_rng(3)
    Ys = [P.Y * (1.0 + 0.01 * rng.standard_normal(P.nobs)) for _ in range(30)]
    out = []
    for lazy in (False, True):
        ctx = B.from_problem(P, prec)
        if lazy:
            ctx.m2m_set_lazy_update(True)
        recs = []
        for Y in Ys:
            ctx.m2m_set_targets(Y, P.sigma)
            ctx.m2m_step(1)
            recs.append(ctx.m2m_get_record())
        y, D, Dt = ctx.m2m_get_obs()
        out.append((recs, y, Dt, ctx.state()))
        ctx.m2m_free()
    (r0, y0, d0, g0), (r1, y1, d1, g1) = out
    # FP32C: exact histograms, so chi^2 and everything else is bit-identical;
    # S and sum w are per-thread sums whose terms the fused pass forms from
    # the update it has just made, the plain pass from the stored weight.
    # FP64 histograms are double sums in atomic order: rounding-level apart.
    # S = -sum w ln(w/w_hat) takes ln w from the fast float logarithm
    # (absolute error < 2^-21.4) on both sides, in other arguments: the two
    # agree to 2e-6 sum w; F = -chi^2/2 + mu S follows.
    exact = prec == "fp32c"
    for a, b in zip(r0, r1):
        assert a["step"] == b["step"]
        for k in ("chi2", "chi2_raw", "max_abs_dt"):
            if exact:
                assert a[k] == b[k], k
            else:
                assert b[k] == pytest.approx(a[k], rel=1e-9), k
        assert b["sum_w"] == pytest.approx(a["sum_w"], rel=1e-6)
        tol_s = 2e-6 * a["sum_w"] if exact else 1e-12 * a["sum_w"]
        assert abs(b["S"] - a["S"]) <= tol_s
        assert abs(b["F"] - a["F"]) <= P.mu * tol_s + 1e-9 * abs(a["F"])
    if exact:
        assert np.array_equal(y0, y1) and np.array_equal(d0, d1)
    else:
        np.testing.assert_allclose(y1, y0, rtol=1e-10, atol=1e-14 * np.abs(y0).max())
        np.testing.assert_allclose(d1, d0, rtol=1e-8, atol=1e-10)
    for k in KEYS:
        if exact or k not in ("w", "what"):
            assert np.array_equal(g0[k], g1[k]), k
        else:
            np.testing.assert_allclose(g1[k], g0[k], rtol=1e-10)


def test_pending_update_is_applied_before_state_reads_and_changes():
    P = _problem("moving-priors", 12007, "fp32c")
    ref = B.from_problem(P, "fp32c")
    lz = B.from_problem(P, "fp32c")
    lz.m2m_set_lazy_update(True)
    ref.m2m_step(3)
    lz.m2m_step(3)
    # the caller's weights still lack the last update ...
    w_ref, w_lz = _raw(ref)["w"], _raw(lz)["w"]
    assert not np.array_equal(w_ref, w_lz)
    # ... which m2m_finish_update applies
    lz.m2m_finish_update()
    assert np.array_equal(_raw(lz)["w"], w_ref)
    lz.m2m_finish_update()                       # nothing pending: no change
    assert np.array_equal(_raw(lz)["w"], w_ref)
    # push, observe, update and priors each apply a pending update first
    for call in (lambda c: c.m2m_push(2), lambda c: c.m2m_observe(1),
                 lambda c: c.m2m_update_weights(), lambda c: c.m2m_priors()):
        ref.m2m_step(2)
        lz.m2m_step(2)
        call(ref)
        call(lz)
        a, b = _raw(ref), _raw(lz)
        for k in KEYS:
            assert np.array_equal(a[k], b[k]), k
    # turning lazy updates off applies the pending one
    ref.m2m_step(4)
    lz.m2m_step(4)
    lz.m2m_set_lazy_update(False)
    a, b = _raw(ref), _raw(lz)
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k
    ref.m2m_free()
    lz.m2m_free()


def test_async_record_is_the_synchronous_record():
    import ctypes
    P = _problem("moving-priors", 12007, "fp32c")
    ctx = B.from_problem(P, "fp32c")
    ctx.m2m_set_lazy_update(True)
    rsz = ctypes.sizeof(B.m2m_record)
    buf = torch.empty(2 * rsz, dtype=torch.uint8, pin_memory=True)
    ptr = [buf.data_ptr(), buf.data_ptr() + rsz]
    ev = torch.cuda.Event()
    for t in range(30):
        ctx.m2m_step(1)
        ctx.m2m_get_record_async(ptr[t % 2])
        ev.record(torch.cuda.current_stream())
        ev.synchronize()
        rec = B.m2m_record.from_address(ptr[t % 2]).as_dict()
        assert rec["step"] == t + 1
        assert rec == ctx.m2m_get_record()
    ctx.m2m_free()
