"""The device generator of the seeing draws (Philox4x32-10), through the
C-ABI: the published known-answer vectors, and the oracle's words on a
spread of counters and keys."""
import numpy as np
import pytest

from oracle import philox as PH
from test_oracle_pins import philox_kat

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_6403_gb300 import m2m as B  # noqa: E402


def test_device_philox_reproduces_the_known_answer_vectors():
    rows = philox_kat()
    c = np.array([r[0] for r in rows], dtype=np.uint32)
    k = np.array([r[1] for r in rows], dtype=np.uint32)
    got = B.m2m_philox4x32_10(c, k)
    assert got.tolist() == [r[2] for r in rows]


def test_device_philox_equals_the_oracle_on_random_counters():
    rng = np.random.default_rng(17)
    n = 100_003
    c = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    k = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    got = B.m2m_philox4x32_10(c, k)
    # the oracle takes one key per call: every 997th draw with its own key,
    # then all draws under the key (0, 0) as one array
    for i in range(0, n, 997):
        ref = PH.philox4x32_10(c[i, 0], c[i, 1], c[i, 2], c[i, 3], int(k[i, 0]), int(k[i, 1]))
        assert [int(v) for v in ref] == got[i].tolist()
    k0 = np.zeros_like(k)
    got0 = B.m2m_philox4x32_10(c, k0)
    ref0 = np.stack(PH.philox4x32_10(c[:, 0], c[:, 1], c[:, 2], c[:, 3], 0, 0), axis=1)
    assert np.array_equal(got0, ref0)
