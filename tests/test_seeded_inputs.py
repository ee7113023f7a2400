"""The PyTorch copy of the seeded generator (used for workloads whose fields
take gigabytes) reproduces the NumPy one: the same SplitMix64 words and
uniforms bit for bit, the complex Gaussians to float64 rounding, and the
complex64 fields the kernels receive equal up to a rare last-bit difference."""
import numpy as np
import pytest

import seeded_inputs as S

torch = pytest.importorskip("torch")


def test_torch_uniforms_match_numpy_bits():
    idx = np.arange(12345, 12345 + 5000, dtype=np.uint64)
    want = S.splitmix64(1005, idx)
    z = torch.from_numpy(idx.astype(np.int64))
    g = S._u64_as_i64(0x9E3779B97F4A7C15)
    m1, m2 = S._u64_as_i64(0xBF58476D1CE4E5B9), S._u64_as_i64(0x94D049BB133111EB)
    w = S._u64_as_i64(1005) + (z + 1) * g
    w = (w ^ S._shr(w, 30)) * m1
    w = (w ^ S._shr(w, 27)) * m2
    w = w ^ S._shr(w, 31)
    assert np.array_equal(w.numpy().view(np.uint64), want)


@pytest.mark.parametrize("seed,offset", [(7, 0), (1005, 3 * 2 ** 20 + 17), (2 ** 63 + 5, 99)])
def test_torch_gaussians_match_numpy(seed, offset):
    want = S.complex_gaussian(seed, 40000, offset)
    got = S.complex_gaussian_torch(seed, 40000, offset, chunk=7000).numpy()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(want).max())


def test_torch_fields_match_numpy_fields():
    K, n_dir, nrhs = (5, 4, 3), 6, 2
    want = S.field_spectra(1002, n_dir, nrhs, K)[2:5].astype(np.complex64)
    got = S.field_spectra_torch(1002, n_dir, nrhs, K, first=2, count=3).numpy()
    assert got.shape == want.shape
    assert np.count_nonzero(got != want) <= 1
    np.testing.assert_allclose(got, want, rtol=1e-7)
