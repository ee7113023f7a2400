"""Translation operator samples and the FFT'ed operator tensors (Eq. 7, Sec. II.B).

Oracle / test infrastructure only (see package docstring).

For a direction k_p and a box offset Delta = v' - v (integer vector, box edge
a), with R = a |Delta| and R^ = Delta / |Delta|:

    T_p(Delta) = c * sum_{l=0}^{L} (-j)^l (2l + 1) h_l^(2)(k R) P_l(R^ . k_p)

k is the wavenumber of the medium, k = k0 sqrt(eps_r) for a free-space
wavenumber k0 and relative permittivity eps_r (complex with Im eps_r < 0 in a
lossy medium, Sec. III.A.5 and Table IV), and eta = eta0 / sqrt(eps_r).

Readings (the paper is ambiguous or silent here):
  * the sum starts at l = 0 (the printed lower limit 1 drops the monopole term
    that the plane-wave expansion of the Green's function needs);
  * c = 1 by default; c = -k^2 eta / (16 pi^2) ("paper" prefactor) on request;
  * near offsets carry no far interaction and are set to zero: by default the
    Chebyshev shell max_i |d_i| <= 1 ("chebyshev" rule); the paper's rule
    a |Delta| < kappa R^s with kappa = 4 and R^s = a sqrt(3)/2 ("kappa" rule)
    is available; Delta = 0 is always near;
  * circulant embedding (Sec. II.B, n_i = 2 K_i): the operator for offset d_i
    in (-K_i, K_i) is stored at index d_i mod n_i; any index not reached by an
    offset (index K_i when n_i = 2 K_i) is zero.
Arrays here are indexed (x, y, z); the FFT'ed tensor T~_p has shape
(n1, n2, n3) = (2Kx, 2Ky, 2Kz) and T_4D stacks the directions last.
"""
from __future__ import annotations

import numpy as np

from . import fft as _fft
from .special import legendre_all, spherical_hankel2_all

ETA0 = 376.730313668  # free-space wave impedance (ohm), for the "paper" prefactor


def offset_axes(K):
    """Integer offsets per axis: d_i in [-(K_i - 1), K_i - 1]."""
    return [np.arange(-(k - 1), k) for k in K]


def near_mask(dx, dy, dz, rule: str = "chebyshev", kappa: float = 4.0):
    """True where the box pair is near (interaction handled classically, Sec. II.A)."""
    if rule == "chebyshev":
        m = np.maximum(np.maximum(np.abs(dx), np.abs(dy)), np.abs(dz)) <= 1
    elif rule == "kappa":
        # a |Delta| < kappa * a sqrt(3)/2  <=>  |Delta|^2 < (kappa sqrt(3)/2)^2
        m = (dx * dx + dy * dy + dz * dz) < (kappa * np.sqrt(3.0) / 2.0) ** 2
    else:
        raise ValueError(f"unknown near rule {rule!r}")
    return m | ((dx == 0) & (dy == 0) & (dz == 0))


def medium_wavenumber(k0: float, eps_r: complex = 1.0) -> complex:
    """k = k0 sqrt(eps_r), principal root (Im k <= 0 for Im eps_r <= 0)."""
    eps = complex(eps_r)
    return k0 * np.sqrt(eps) if eps.imag != 0 else k0 * np.sqrt(eps.real)


def prefactor_value(k0: float, kind: str = "unit", eps_r: complex = 1.0) -> complex:
    if kind == "unit":
        return 1.0
    if kind == "paper":
        k = medium_wavenumber(k0, eps_r)
        eta = ETA0 / np.sqrt(complex(eps_r)) if complex(eps_r).imag != 0 else ETA0 / np.sqrt(complex(eps_r).real)
        return -(k ** 2) * eta / (16.0 * np.pi ** 2)
    raise ValueError(f"unknown prefactor {kind!r}")


def operator_at(khat, dx, dy, dz, a: float, k0: float, L: int,
                near_rule: str = "chebyshev", prefactor: str = "unit",
                kappa: float = 4.0, eps_r: complex = 1.0):
    """T(k, Delta) of Eq. 7 at arbitrary integer offsets (broadcast arrays).

    khat: (3,) unit vector.  Returns complex128 with the offsets' shape.
    """
    dx, dy, dz = np.broadcast_arrays(np.asarray(dx), np.asarray(dy), np.asarray(dz))
    d2 = (dx * dx + dy * dy + dz * dz).astype(np.int64)
    near = near_mask(dx, dy, dz, near_rule, kappa)
    out = np.zeros(dx.shape, dtype=np.complex128)
    far = ~near
    if not np.any(far):
        return out
    d2f = d2[far]
    # Hankel values depend only on |Delta|^2: evaluate once per distinct value
    uniq, inv = np.unique(d2f, return_inverse=True)
    kr = medium_wavenumber(k0, eps_r) * a * np.sqrt(uniq.astype(np.float64))
    h = spherical_hankel2_all(L, kr)[:, inv]                  # (L+1, n_far)
    dist = np.sqrt(d2f.astype(np.float64))
    cosang = (khat[0] * dx[far] + khat[1] * dy[far] + khat[2] * dz[far]) / dist
    P = legendre_all(L, cosang)                                # (L+1, n_far)
    l = np.arange(L + 1)
    coef = ((-1j) ** l) * (2 * l + 1)
    out[far] = prefactor_value(k0, prefactor, eps_r) * np.einsum("l,ln,ln->n", coef, h, P)
    return out


def operator_grid(khat, K, a, k0, L, near_rule="chebyshev", prefactor="unit", kappa=4.0, eps_r=1.0):
    """T_p(Delta) on the full offset grid, shape (2Kx-1, 2Ky-1, 2Kz-1), index d + K - 1."""
    ax = offset_axes(K)
    dx, dy, dz = np.meshgrid(*ax, indexing="ij")
    return operator_at(khat, dx, dy, dz, a, k0, L, near_rule, prefactor, kappa, eps_r)


def embed(Tgrid, K, n):
    """Circulant embedding of the offset grid into an n1 x n2 x n3 array (Sec. II.B)."""
    out = np.zeros(tuple(n), dtype=np.complex128)
    ix = [np.arange(-(k - 1), k) % nn for k, nn in zip(K, n)]
    out[np.ix_(*ix)] = Tgrid
    return out


def fft_operator(khat, K, n, a, k0, L, near_rule="chebyshev", prefactor="unit", kappa=4.0, eps_r=1.0):
    """FFT'ed translation operator T~_p = FFT3(embed(T_p)) for one direction."""
    T = operator_grid(khat, K, a, k0, L, near_rule, prefactor, kappa, eps_r)
    return _fft.fftn(embed(T, K, n), axes=(0, 1, 2))
