"""The oracle's own discrete Fourier transform (the FFT operator of Eq. 5).

Oracle / test infrastructure only (see package docstring).

Convention (the paper does not state one; the translated fields do not depend
on it as long as the operator and the fields use the same forward transform):
  forward  X[k] = sum_n x[n] exp(-2 pi i n k / N)      (unnormalised)
  inverse  x[n] = (1/N) sum_k X[k] exp(+2 pi i n k / N)

Algorithm: recursive decimation-in-time Cooley-Tukey over the smallest factor
p in {2, 3, 5, 7} of N: x is split into the p subsequences x[p t + s], each is
transformed, and X[k] = sum_s exp(-+2 pi i s k / N) X_s[k mod N/p].  A length
with no factor in {2, 3, 5, 7} is transformed as a plain DFT matrix product.
Vectorised over every axis but the transformed one.
"""
from __future__ import annotations

import numpy as np

_RADICES = (2, 3, 5, 7)


def _smallest_radix(n: int) -> int:
    for p in _RADICES:
        if n % p == 0:
            return p
    return n


def _dft_last(x: np.ndarray, sign: int) -> np.ndarray:
    n = x.shape[-1]
    k = np.arange(n)
    W = np.exp(sign * 2j * np.pi * np.outer(k, k) / n)
    return x @ W.T


def _fft_last(x: np.ndarray, sign: int) -> np.ndarray:
    n = x.shape[-1]
    if n == 1:
        return x.astype(np.complex128, copy=True)
    p = _smallest_radix(n)
    if p == n:
        return _dft_last(x, sign)
    m = n // p
    k = np.arange(n)
    out = np.zeros(x.shape, dtype=np.complex128)
    for s in range(p):
        sub = _fft_last(x[..., s::p], sign)            # length m
        out += np.exp(sign * 2j * np.pi * s * k / n) * sub[..., k % m]
    return out


def fft(x: np.ndarray, axis: int = -1) -> np.ndarray:
    """Forward unnormalised DFT along one axis."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    return np.moveaxis(_fft_last(x, -1), -1, axis)


def ifft(x: np.ndarray, axis: int = -1) -> np.ndarray:
    """Inverse DFT along one axis, normalised by 1/N."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    return np.moveaxis(_fft_last(x, +1) / n, -1, axis)


def fftn(x: np.ndarray, axes=(-3, -2, -1)) -> np.ndarray:
    """Forward multi-dimensional DFT as successive 1D transforms."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in axes:
        out = fft(out, ax)
    return out


def ifftn(x: np.ndarray, axes=(-3, -2, -1)) -> np.ndarray:
    """Inverse multi-dimensional DFT (normalised) as successive 1D transforms."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in axes:
        out = ifft(out, ax)
    return out


def naive_dft(x: np.ndarray, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """O(N^2) DFT by its definition, used to pin `fft` on small sizes."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    out = _dft_last(x, +1 if inverse else -1)
    if inverse:
        out = out / n
    return np.moveaxis(out, -1, axis)
