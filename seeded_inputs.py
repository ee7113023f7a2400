"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only random-number generation and shape bookkeeping; none of
the translation method's arithmetic lives here.  Both the CPU oracle and the
GPU path take their field spectra from these functions, so they see the same
bits.

Generator (published definitions, written out here):
  * SplitMix64 (Steele, Lea & Flood 2014, as given by Vigna): the k-th output
    for a seed s is mix(s + (k + 1) * 0x9E3779B97F4A7C15) with
    mix(z) = z ^ (z >> 31) after z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9,
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB (all modulo 2**64).
    Used in counter mode: element i of a stream draws outputs 2i and 2i + 1.
  * Uniforms: u = ((z >> 11) + 1) * 2**-53, which lies in (0, 1].
  * Box-Muller: for uniforms u1, u2 the complex value
    sqrt(-ln u1) * (cos 2 pi u2 + j sin 2 pi u2) has real and imaginary parts
    that are independent N(0, 1/2), i.e. a unit-variance circular complex
    Gaussian.

Field layout used everywhere in this project: a complex array of shape
(n_dir, 2, nrhs, Kz, Ky, Kx) -- direction, polarisation (theta, phi),
right-hand side, then the box grid with x fastest.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for the given 0-based counters (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in (0, 1] from SplitMix64 outputs."""
    z = splitmix64(seed, counters)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def complex_gaussian(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` circular complex Gaussians (E|z|^2 = 1), element i = offset + i."""
    idx = np.arange(offset, offset + count, dtype=np.uint64)
    u1 = uniform01(seed, np.uint64(2) * idx)
    u2 = uniform01(seed, np.uint64(2) * idx + np.uint64(1))
    rad = np.sqrt(-np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang) + 1j * rad * np.sin(ang)


def field_spectra(seed: int, n_dir: int, nrhs: int, K: tuple[int, int, int],
                  dtype=np.complex128) -> np.ndarray:
    """Aggregated theta/phi box spectra A_v(k_p) for every direction.

    Shape (n_dir, 2, nrhs, Kz, Ky, Kx) with K = (Kx, Ky, Kz).  Dense i.i.d.
    circular complex Gaussians stand in for the aggregations of a meshed
    structure (no mesh is available); every box is occupied.
    """
    Kx, Ky, Kz = K
    shape = (n_dir, 2, nrhs, Kz, Ky, Kx)
    vals = complex_gaussian(seed, int(np.prod(shape)))
    return vals.reshape(shape).astype(dtype)


def field_spectra_rows(seed: int, n_dir: int, nrhs: int, K: tuple[int, int, int],
                       fields: np.ndarray) -> np.ndarray:
    """Only the listed flat field indices of `field_spectra` (same values).

    Field index f = (p * 2 + pol) * nrhs + rhs.  Returns (len(fields), Kz, Ky, Kx)
    complex128.  Lets a check regenerate a few fields of a large workload
    without materialising all of it.
    """
    Kx, Ky, Kz = K
    per = Kx * Ky * Kz
    out = np.empty((len(fields), Kz, Ky, Kx), dtype=np.complex128)
    for i, f in enumerate(np.asarray(fields, dtype=np.int64)):
        out[i] = complex_gaussian(seed, per, offset=int(f) * per).reshape(Kz, Ky, Kx)
    return out


def _u64_as_i64(v: int) -> int:
    """The int64 with the same 64 bits as the unsigned value v."""
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def _shr(z, k: int):
    """Logical right shift of int64 words holding uint64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def complex_gaussian_torch(seed: int, count: int, offset: int = 0, device="cpu", chunk: int = 1 << 24):
    """The values of complex_gaussian(seed, count, offset), computed with
    PyTorch int64 / float64 tensor operations on `device` (same SplitMix64
    words, same uniforms, Box-Muller in float64): complex128 tensor.

    For workloads whose fields take gigabytes, where the NumPy generator would
    take minutes.  The integer steps (int64 words with wrap-around products
    and masked shifts standing in for uint64 arithmetic) give the same bits;
    log, cos and sin are the device library's float64 functions, so values may
    differ from NumPy's in the last bit of float64 (and, rarely, one bit of a
    value rounded to complex64)."""
    import torch

    g = _u64_as_i64(0x9E3779B97F4A7C15)
    m1, m2 = _u64_as_i64(0xBF58476D1CE4E5B9), _u64_as_i64(0x94D049BB133111EB)
    s0 = _u64_as_i64(seed)
    out = torch.empty(count, dtype=torch.complex128, device=device)

    def words(ctr):
        z = s0 + (ctr + 1) * g
        z = (z ^ _shr(z, 30)) * m1
        z = (z ^ _shr(z, 27)) * m2
        return z ^ _shr(z, 31)

    for c0 in range(0, count, chunk):
        n = min(chunk, count - c0)
        idx = torch.arange(offset + c0, offset + c0 + n, dtype=torch.int64, device=device)
        u1 = (_shr(words(2 * idx), 11).to(torch.float64) + 1.0) * (2.0 ** -53)
        u2 = (_shr(words(2 * idx + 1), 11).to(torch.float64) + 1.0) * (2.0 ** -53)
        rad = torch.sqrt(-torch.log(u1))
        ang = 2.0 * np.pi * u2
        out[c0:c0 + n] = torch.complex(rad * torch.cos(ang), rad * torch.sin(ang))
    return out


def field_spectra_torch(seed: int, n_dir: int, nrhs: int, K: tuple[int, int, int], first: int = 0,
                        count: int | None = None, device="cpu", dtype=None):
    """Directions first .. first + count - 1 of field_spectra(seed, n_dir, nrhs,
    K), generated on `device` one direction at a time by complex_gaussian_torch
    and stored as `dtype` (default complex64): shape (count, 2, nrhs, Kz, Ky, Kx)."""
    import torch

    Kx, Ky, Kz = K
    count = n_dir - first if count is None else count
    dtype = torch.complex64 if dtype is None else dtype
    per_dir = 2 * nrhs * Kx * Ky * Kz
    out = torch.empty((count, 2, nrhs, Kz, Ky, Kx), dtype=dtype, device=device)
    for q in range(count):
        vals = complex_gaussian_torch(seed, per_dir, (first + q) * per_dir, device=device)
        out[q] = vals.reshape(2, nrhs, Kz, Ky, Kx).to(dtype)
    return out


def shell_occupancy(K: tuple[int, int, int], thickness: float = 1.0) -> np.ndarray:
    """Box occupancy of a surface mesh of the sphere inscribed in the box
    grid: a (Kz, Ky, Kx) boolean array, True where a box centre lies within
    `thickness` box edges of the sphere.  Stands in for the shell of boxes a
    meshed sphere occupies (its interior boxes are empty)."""
    Kx, Ky, Kz = K
    z, y, x = np.meshgrid(np.arange(Kz), np.arange(Ky), np.arange(Kx), indexing="ij")
    c = [(k - 1) / 2.0 for k in (Kx, Ky, Kz)]
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    R = min(Kx, Ky, Kz) / 2.0 - 0.5
    return np.abs(r - R) <= thickness


# Workloads (box grids, multipole counts, formats) of the synthetic benchmark
# suite.  All use box edge a = 0.5 wavelengths with wavelength 1 (k0 = 2 pi),
# the Chebyshev near rule max|d_i| <= 1 and N_phi = 2(L+1).
WORKLOADS = {
    "c128_plain_8cube_L5": dict(K=(8, 8, 8), L=5, nrhs=1, fmt="none", decomp="none",
                                 tol=0.0, prec="c128", seed=1001),
    "tucker3d_32cube_L8": dict(K=(32, 32, 32), L=8, nrhs=4, fmt="3d", decomp="tucker",
                               tol=1e-4, prec="c64_3xtf32", seed=1002),
    "tt4d_64cube_L10": dict(K=(64, 64, 64), L=10, nrhs=1, fmt="4d", decomp="tt",
                            tol=1e-3, prec="c64_bf16x3", seed=1003),
    "htucker4d_64cube_L10": dict(K=(64, 64, 64), L=10, nrhs=1, fmt="4d", decomp="htucker",
                                 tol=1e-3, prec="c64_bf16x3", seed=1003),
    "tucker3d_128x128x32_L6": dict(K=(128, 128, 32), L=6, nrhs=16, fmt="3d", decomp="tucker",
                                   tol=1e-4, prec="c64_3xtf32", seed=1005),
}
