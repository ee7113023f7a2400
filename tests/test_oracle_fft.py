"""Pins for the oracle's own FFT (the transform of Eq. 5): naive DFT and numpy.fft."""
import numpy as np
import pytest

from oracle import fft as F


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 14, 15, 16, 21, 24, 30, 35, 49, 64, 11, 13])
def test_fft_vs_naive_and_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    X = F.fft(x)
    np.testing.assert_allclose(X, F.naive_dft(x), rtol=0, atol=1e-12 * max(1, n))
    np.testing.assert_allclose(X, np.fft.fft(x), rtol=0, atol=1e-12 * max(1, n))
    np.testing.assert_allclose(F.ifft(X), x, atol=1e-13 * max(1, n))
    np.testing.assert_allclose(F.ifft(X), np.fft.ifft(X), atol=1e-13 * max(1, n))


def test_fftn_axes_and_roundtrip():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((4, 6, 8)) + 1j * rng.standard_normal((4, 6, 8))
    np.testing.assert_allclose(F.fftn(x, axes=(0, 1, 2)), np.fft.fftn(x), atol=1e-11)
    np.testing.assert_allclose(F.ifftn(F.fftn(x)), x, atol=1e-13)


def test_naive_dft_definition_small():
    # X[k] = sum_n x[n] e^{-2 pi i n k / N} written out for N = 3
    x = np.array([1.0, 2.0j, -0.5 + 0.25j])
    w = np.exp(-2j * np.pi / 3)
    ref = np.array([x[0] + x[1] + x[2], x[0] + x[1] * w + x[2] * w ** 2, x[0] + x[1] * w ** 2 + x[2] * w ** 4])
    np.testing.assert_allclose(F.naive_dft(x), ref, atol=1e-15)
