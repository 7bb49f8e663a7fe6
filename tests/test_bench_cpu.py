"""The bench's roofline bookkeeping on CPU: the dominant kernel and its
per-launch time from the library's timing record, the algorithmic bytes
per particle-step, and the measured DRAM traffic, which is reported only
for the device sources and particle count it was captured on."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod_cpu", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _timing(steps_launches, steps_ms, steps_steps, pass_launches=0, pass_ms=0.0):
    z = {k: 0 for k in ("step_upd", "step", "residual", "update", "prior", "other", "sh", "steps")}
    launches, ms, steps = dict(z), {k: 0.0 for k in z}, dict(z)
    launches["steps"], ms["steps"], steps["steps"] = steps_launches, steps_ms, steps_steps
    launches["step_upd"], ms["step_upd"] = pass_launches, pass_ms
    return {"launches": launches, "ms": ms, "steps": steps}


def test_algorithmic_bytes_per_particle_step(bench):
    # FP32C: x, v read and written (6 floats each way), w read and written
    # (double), w_hat read (double); FP64: the same with double positions
    assert bench.BYTES_PER_PARTICLE_FP32C == 2 * 6 * 4 + 2 * 8 + 8
    assert bench.BYTES_PER_PARTICLE_FP64 == 2 * 6 * 8 + 2 * 8 + 8


def test_dominant_kernel_is_the_persistent_launch_when_it_ran(bench):
    name, ms, spl = bench.dominant(_timing(4, 7.4, 100, pass_launches=3, pass_ms=0.3), "k_pass")
    assert name.startswith("k_steps") and ms == pytest.approx(7.4 / 4) and spl == pytest.approx(25.0)
    name, ms, spl = bench.dominant(_timing(0, 0.0, 0, pass_launches=10, pass_ms=0.8), "k_pass")
    assert name == "k_pass" and ms == pytest.approx(0.08) and spl == 1.0


def test_measured_traffic_only_for_the_captured_sources_and_size(bench, tmp_path, monkeypatch):
    prof = {"k_steps": {"src_sha": "abc", "n": 1000, "dram_bytes_per_step": 123.0},
            "k_pass": {"src_sha": "abc", "n": 1000, "dram_bytes_per_step": 77.0}}
    p = tmp_path / "prof.json"
    p.write_text(json.dumps(prof))
    monkeypatch.setattr(bench, "PROFILE_JSON", str(p))
    monkeypatch.setattr(bench, "src_hash", lambda: "abc")
    assert bench.measured_traffic("k_steps (persistent)", 1000, 20.0) == pytest.approx(2460.0)
    assert bench.measured_traffic("k_pass (steady)", 1000, 1.0) == pytest.approx(77.0)
    assert bench.measured_traffic("k_steps (persistent)", 2000, 20.0) is None      # another size
    monkeypatch.setattr(bench, "src_hash", lambda: "changed")
    assert bench.measured_traffic("k_steps (persistent)", 1000, 20.0) is None      # other device code
    monkeypatch.setattr(bench, "PROFILE_JSON", str(tmp_path / "missing.json"))
    assert bench.measured_traffic("k_pass", 1000, 1.0) is None


def test_committed_capture_names_its_command_and_size(bench):
    with open(bench.PROFILE_JSON) as f:
        prof = json.load(f)
    for key in ("k_steps", "k_pass"):
        e = prof[key]
        assert e["n"] == 4_000_000 and e["dram_bytes_per_step"] > 0
        assert "--clock-control none" in e["command"]
        # the traffic per step against the algorithmic bytes of a step
        ratio = e["dram_bytes_per_step"] / (bench.BYTES_PER_PARTICLE_FP32C * e["n"])
        assert 0.5 < ratio < 1.2
