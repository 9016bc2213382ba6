"""The seeded input generator: the vectorised numpy stream against a scalar
SplitMix64 (Steele, Lea and Flood 2014: state += golden gamma, then the
variant-13 mix), and the torch twin (run here on the CPU) against numpy, bit
for bit on coordinates and to float rounding on values."""
import numpy as np
import pytest

import synthdata as S

torch = pytest.importorskip("torch")


def _splitmix_scalar(key, i):
    z = (key + (i + 1) * S.GAMMA) & S.MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & S.MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & S.MASK64
    return z ^ (z >> 31)


def test_first_splitmix_output_of_seed_zero():
    # the published generator's first output from state 0 (gamma added first)
    assert _splitmix_scalar(0, 0) == 0xE220A8397B1DCDAF


def test_vectorised_stream_matches_scalar_definition():
    key = S.stream_key(7, S.S_X * 8)
    idx = np.arange(1000, 1064, dtype=np.uint64)
    got = S._u64_np(key, idx)
    want = np.array([_splitmix_scalar(key, int(i)) for i in idx], dtype=np.uint64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_torch_twin_uniforms_are_bit_identical(dtype):
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    a = S.uniform_np(3, 11, 5000, 4096, dtype=dtype)
    b = S.uniform_torch(3, 11, 5000, 4096, tdt, "cpu").numpy()
    assert np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() < 1.0


def test_torch_twin_workload_matches_numpy():
    rec = S.config("matern2d_1e9", n=100_000)
    x, y, _ = S.make_np(rec)
    xt, yt = S.make_torch(rec, "cpu", chunk=30_000)
    assert np.array_equal(x, xt.numpy())
    assert np.abs(y - yt.numpy()).max() <= 1e-5 * np.abs(y).max()


def test_points_are_in_the_unit_cube_and_uniform():
    rec = S.config("matern2d", n=200_000)
    x, _, _ = S.make_np(rec)
    assert x.min() >= 0.0 and x.max() <= 1.0
    hist, _ = np.histogram(x[:, 0], bins=20, range=(0, 1))
    # 20 bins of 10000 expected: a 6-sigma band of the binomial count
    assert np.abs(hist - 10_000).max() <= 6 * np.sqrt(10_000 * 0.95)
