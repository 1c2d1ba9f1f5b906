"""The torch form of the input generator (synth.*_torch) reproduces the numpy one:
the uniforms bit for bit (same SplitMix64 words), the normals to rounding."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("seed", [0, 7, 2 ** 40 + 5, 0xFFFFFFFF])
def test_uniforms_bitwise(seed):
    a = synth.uniform01(seed, 4097)
    b = synth.uniform01_torch(seed, 4097).numpy()
    assert np.array_equal(a, b)


def test_normal_rhs_matches_host_generator():
    a = synth.rhs_normal(128, 123)
    b = synth.rhs_normal_torch(128, 123).numpy()
    assert np.max(np.abs(a - b)) <= 1e-14
    assert np.all(b[0, :] == 0) and np.all(b[-1, :] == 0) and np.all(b[:, 0] == 0) and np.all(b[:, -1] == 0)
    out = torch.full((129, 129), 5.0, dtype=torch.float64)
    synth.rhs_normal_torch(128, 123, out=out)
    assert torch.equal(out, torch.from_numpy(b))
