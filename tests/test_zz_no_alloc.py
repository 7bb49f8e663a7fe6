"""m2m_observe_static: the observe entry point for callers that cannot
allocate device memory (under an external allocator that owns all device
memory, allocator-free deployments, code that must not trigger the
implicit synchronisation of cudaMalloc/cudaFree).  Its scratch is one
fixed array in the library, shared by every call; this file checks,
through the C-ABI, that two calls in a row reproduce the context-based
m2m_observe and the oracle's observe, that the shared totals are cleared
between calls, and that sizes beyond the fixed capacity are refused.
Collected last on purpose."""
import numpy as np
import pytest

from oracle import m2m as O
from paper_1207_6403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402


def _problem():
    P = I.make_problem("flat-log", n=50_003, precision="fp32c")
    Y = O.observe(*P.target_pos, *P.target_vel, P.target_w, P.obs, P.incl_sin, P.incl_cos)
    # weights 2^-16: their sum (0.763) is exact, so the context's fixed-point
    # scale (from its sum of weights) is known to the test
    w = np.full(P.n, 2.0 ** -16)
    return I.Problem(**{**P.with_targets(Y).__dict__, "w0": w, "what0": w.copy()})


def _close(a, b, sigma, tol=1e-5):
    scale = np.maximum(np.maximum(np.abs(b), sigma / 0.02), 1e-300)
    assert np.max(np.abs(a - b) / scale) <= tol


def test_static_observe_matches_context_observe_twice():
    P = _problem()
    ctx = B.from_problem(P, "fp32c")
    y_ctx, _, _ = ctx.m2m_get_obs()            # the context's initial scatter
    t = ctx.t
    out = torch.empty(P.nobs, dtype=torch.float64, device=t["w"].device)
    W = float(np.sum(P.w0))
    # the oracle's observe of the same (float32) state, in float64
    h = {k: v.cpu().numpy() for k, v in t.items()}
    y_orc = O.observe(h["x"], h["y"], h["z"], h["vx"], h["vy"], h["vz"], h["w"], P.obs, P.incl_sin, P.incl_cos)
    for _ in range(2):                          # two calls in a row
        out.fill_(-1.0)
        B.m2m_observe_static((t["x"], t["y"], t["z"]), (t["vx"], t["vy"], t["vz"]), t["w"], P.obs,
                             P.incl_sin, P.incl_cos, W, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        _close(got, y_ctx, P.sigma)
        _close(got, y_orc, P.sigma)
        # weight_scale = the context's sum of weights: the same fixed-point
        # scale, so the same exact integer sums
        assert np.array_equal(got, y_ctx)
    # a third call with doubled weights: the shared totals start from zero
    w2 = t["w"] * 2.0
    B.m2m_observe_static((t["x"], t["y"], t["z"]), (t["vx"], t["vy"], t["vz"]), w2, P.obs,
                         P.incl_sin, P.incl_cos, 2.0 * W, out)
    torch.cuda.synchronize()
    _close(out.cpu().numpy(), 2.0 * y_ctx, 2.0 * P.sigma)
    ctx.m2m_free()


def test_static_observe_refuses_sizes_beyond_capacity():
    P = _problem()
    big = [I.ObservableSet("grid", "mass", I.uniform_edges(100, -3, 3), I.uniform_edges(100, -3, 3))]
    t = {k: torch.zeros(16, dtype=torch.float32, device="cuda") for k in ("x", "y", "z", "vx", "vy", "vz")}
    w = torch.full((16,), 1.0 / 16, dtype=torch.float64, device="cuda")
    out = torch.empty(10000, dtype=torch.float64, device="cuda")
    with pytest.raises(B.M2MError) as e:
        B.m2m_observe_static((t["x"], t["y"], t["z"]), (t["vx"], t["vy"], t["vz"]), w, big, 0.0, 1.0, 1.0, out)
    assert e.value.code == -1 and "capacity" in str(e.value)
