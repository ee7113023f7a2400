"""Special functions of Eq. 7: spherical Hankel h_l^(2) and Legendre P_l.

Oracle / test infrastructure only (see package docstring).

h_l^(2)(x) = j_l(x) - i y_l(x) for real x > 0.  Each part is computed in its
stable direction:
  * y_l by upward recurrence from the closed forms of y_0 and y_1;
  * j_l by Miller's downward recurrence, normalised with the identity
    sum_{l>=0} (2l + 1) j_l(x)^2 = 1, which holds for every x and so avoids
    the cancellation that a j_0 = sin(x)/x normalisation suffers at x = m pi.
Both families satisfy f_{l+1}(x) = (2l + 1)/x f_l(x) - f_{l-1}(x).
For a complex argument z (a lossy medium, Sec. III.A.5: Im z < 0) h_l^(2) is
taken from its terminating series in 1/z,
    h_l^(2)(z) = e^{-iz} sum_{k=0}^{l} (-i)^{k-l-1} a_k(l) / z^{k+1},
    a_k(l) = (l + k)! / (2^k k! (l - k)!),
which never forms j_l and y_l (both of size e^{|Im z|} there, cancelling).
P_l(t) by Bonnet's recurrence (l + 1) P_{l+1} = (2l + 1) t P_l - l P_{l-1}.
"""
from __future__ import annotations

import math

import numpy as np


def spherical_yn_all(lmax: int, x: np.ndarray) -> np.ndarray:
    """y_0..y_lmax at x (> 0); returns shape (lmax + 1,) + x.shape."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((lmax + 1,) + x.shape)
    out[0] = -np.cos(x) / x
    if lmax >= 1:
        out[1] = -np.cos(x) / (x * x) - np.sin(x) / x
    for l in range(1, lmax):
        out[l + 1] = (2 * l + 1) / x * out[l] - out[l - 1]
    return out


def spherical_jn_all(lmax: int, x: np.ndarray) -> np.ndarray:
    """j_0..j_lmax at x (> 0) by Miller's downward recurrence."""
    x = np.asarray(x, dtype=np.float64)
    flat = x.ravel()
    xmax = float(np.max(flat)) if flat.size else 1.0
    lstart = int(lmax + 40 + 2 * np.ceil(xmax))
    f = np.zeros((lstart + 2, flat.size))
    # start small but far from underflow: the normalisation sums f^2, and a
    # start near 1e-200 leaves f^2 subnormal when the recurrence grows little
    # (small lmax, moderate x); rescale whenever a value passes 1e100
    f[lstart] = 1e-100
    for l in range(lstart, 0, -1):
        f[l - 1] = (2 * l + 1) / flat * f[l] - f[l + 1]
        big = np.abs(f[l - 1]) > 1e100
        if np.any(big):
            f[:, big] *= 1e-100
    ls = np.arange(lstart + 2, dtype=np.float64)[:, None]
    norm = np.sqrt(np.sum((2 * ls + 1) * f * f, axis=0))
    j = f[: lmax + 1] / norm
    # fix the overall sign against whichever closed form is better conditioned
    j0 = np.sin(flat) / flat
    j1 = np.sin(flat) / (flat * flat) - np.cos(flat) / flat
    s0 = np.sign(j[0] * j0)
    s1 = np.sign(f[1] * j1)
    sign = np.where(np.abs(j0) >= np.abs(j1), s0, s1)
    j = j * sign
    return j.reshape((lmax + 1,) + x.shape)


def spherical_hankel2_series(lmax: int, z: np.ndarray) -> np.ndarray:
    """h_0^(2)..h_lmax^(2) at complex z (Re z > 0) from the terminating series."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.empty((lmax + 1,) + z.shape, dtype=np.complex128)
    e = np.exp(-1j * z)
    for l in range(lmax + 1):
        acc = np.zeros(z.shape, dtype=np.complex128)
        for k in range(l + 1):
            a_k = math.factorial(l + k) / (2.0 ** k * math.factorial(k) * math.factorial(l - k))
            acc = acc + ((-1j) ** (k - l - 1)) * a_k / z ** (k + 1)
        out[l] = e * acc
    return out


def spherical_hankel2_all(lmax: int, x: np.ndarray) -> np.ndarray:
    """h_l^(2)(x) = j_l(x) - i y_l(x) for l = 0..lmax (complex128); complex x
    goes through the terminating series."""
    if np.iscomplexobj(x):
        return spherical_hankel2_series(lmax, x)
    return spherical_jn_all(lmax, x) - 1j * spherical_yn_all(lmax, x)


def legendre_all(lmax: int, t: np.ndarray) -> np.ndarray:
    """P_0..P_lmax at t via Bonnet's recurrence; shape (lmax + 1,) + t.shape."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty((lmax + 1,) + t.shape)
    out[0] = 1.0
    if lmax >= 1:
        out[1] = t
    for l in range(1, lmax):
        out[l + 1] = ((2 * l + 1) * t * out[l] - l * out[l - 1]) / (l + 1)
    return out
