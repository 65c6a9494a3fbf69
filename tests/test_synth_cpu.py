"""CPU checks of the seeded input generator (paper_1803_00005_gb300/synth.py), which both the CUDA
path's tests and the oracle's tests draw from: its cost volume follows the truncated colour +
gradient recipe that the oracle's cost_volume implements (pinned in test_oracle_pins.py), its
bfloat16 rounding agrees with torch's, and its scenes are deterministic per seed and in range."""
import numpy as np
import pytest

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_cost_volume_follows_the_oracle_recipe(dtype):
    left, right, _ = synth.stereo_pair(41, 29, 9, seed=11)
    V = synth.from_dtype(synth.cost_volume(left, right, 9, dtype), dtype)
    ref = O.cost_volume(left, right, 9)
    # one rounding to the storage type apart: half an ulp of that type, plus float64 noise
    mant = {"f32": 23, "f16": 10, "bf16": 7}[dtype]
    tol = np.abs(ref) * 2.0 ** -mant + 1e-12
    assert np.all(np.abs(V - ref) <= tol)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.uniform(0, 0.05, 4000), rng.normal(0, 10, 4000),
                        [0.0, -0.0, 1.0, 2.0 ** -130, 3.0e38]])
    ours = synth.to_dtype(v, "bf16")
    theirs = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(ours, theirs.view(np.uint16))


def test_stereo_pair_deterministic_and_in_range():
    a = synth.stereo_pair(64, 48, 16, seed=1)
    b = synth.stereo_pair(64, 48, 16, seed=1)
    c = synth.stereo_pair(64, 48, 16, seed=2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[0], c[0])
    left, right, disp = a
    assert left.shape == right.shape == (3, 48, 64)
    assert left.min() >= 0.0 and left.max() <= 1.0 and right.min() >= 0.0 and right.max() <= 1.0
    assert disp.min() >= 0 and disp.max() <= 15
    # the right view is made of left-view samples along the same row
    for y in range(48):
        for x in range(64):
            assert any(np.array_equal(right[:, y, x], left[:, y, xs]) for xs in range(x, 64))
