"""Translation stage: B = IFFT(T~_p . FFT(A)) for every field (Eq. 5).

Oracle / test infrastructure only (see package docstring).

Fields use the project layout (n_dir, 2, nrhs, Kz, Ky, Kx) with x fastest;
operators are indexed (x, y, z).  The same T~_p multiplies both polarisations
and every right-hand side of direction p (Sec. II.A: only the theta and phi
components are translated, with the same scalar operator).

Two routes that must agree (Sec. II.A, Eq. 5):
  translate_fft     zero-pad A to n1 x n2 x n3, forward FFT, multiply by T~_p,
                    inverse FFT, keep the K1 x K2 x K3 corner;
  translate_direct  B(v') = sum_v T_p(v' - v) A(v), the Toeplitz sum the FFT
                    route evaluates fast (brute force, small grids only).
"""
from __future__ import annotations

import numpy as np

from . import fft as _fft


def translate_field_fft(That, A_zyx):
    """One field: A (Kz, Ky, Kx) -> B (Kz, Ky, Kx) through the (n1, n2, n3) grid."""
    n = That.shape
    Kz, Ky, Kx = A_zyx.shape
    pad = np.zeros(n, dtype=np.complex128)
    pad[:Kx, :Ky, :Kz] = np.transpose(A_zyx, (2, 1, 0))
    C = _fft.fftn(pad, axes=(0, 1, 2)) * That
    Bfull = _fft.ifftn(C, axes=(0, 1, 2))
    return np.transpose(Bfull[:Kx, :Ky, :Kz], (2, 1, 0))


def translate_fft(Thats, S_in):
    """All fields.  Thats: sequence of n_dir arrays (n1, n2, n3); S_in as above."""
    n_dir = S_in.shape[0]
    out = np.empty(S_in.shape, dtype=np.complex128)
    for p in range(n_dir):
        Th = Thats[p]
        for pol in range(S_in.shape[1]):
            for r in range(S_in.shape[2]):
                out[p, pol, r] = translate_field_fft(Th, S_in[p, pol, r])
    return out


def translate_field_direct(Tgrid, A_zyx):
    """B(v') = sum_v T(v' - v) A(v); Tgrid indexed (d + K - 1) in (x, y, z)."""
    Kz, Ky, Kx = A_zyx.shape
    B = np.zeros((Kz, Ky, Kx), dtype=np.complex128)
    for vz in range(Kz):
        for vy in range(Ky):
            for vx in range(Kx):
                a = A_zyx[vz, vy, vx]
                if a == 0:
                    continue
                # offsets v' - v for all v' at once: index (v' - v) + K - 1
                sub = Tgrid[Kx - 1 - vx: 2 * Kx - 1 - vx,
                            Ky - 1 - vy: 2 * Ky - 1 - vy,
                            Kz - 1 - vz: 2 * Kz - 1 - vz]
                B += a * np.transpose(sub, (2, 1, 0))
    return B


def translate_point_direct(Tfun, A_zyx, vprime):
    """One output box v' = (x, y, z) by the direct sum; Tfun(dx, dy, dz) -> T values."""
    Kz, Ky, Kx = A_zyx.shape
    vz, vy, vx = np.meshgrid(np.arange(Kz), np.arange(Ky), np.arange(Kx), indexing="ij")
    T = Tfun(vprime[0] - vx, vprime[1] - vy, vprime[2] - vz)
    return np.sum(T * A_zyx)
