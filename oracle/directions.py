"""Plane-wave directions on the Ewald sphere (Sec. II.A).

Oracle / test infrastructure only (see package docstring).

The paper samples directions as the Cartesian product of quadrature points in
theta and phi and gives the number of multipoles L as a function of the box
radius and the desired number of accurate digits.  Readings taken here:
  * theta nodes: Gauss-Legendre in x = cos(theta), L + 1 of them;
  * phi nodes: uniform, N_phi = 2(L + 1) by default ("benchmark" rule), or
    N_phi = 2L + 1 ("paper" rule, N_dir = (L+1)(2L+1) as printed in Sec. II.A);
  * ordering: theta-major, p = i * N_phi + j with x_i ascending and
    phi_j = 2 pi j / N_phi;
  * multipole count: L = floor(2kR + (2kR)^(1/3) * 1.8 * digits^(2/3)) with
    R = a sqrt(3) / 2 the radius of the sphere enclosing a box and |k| for a
    complex wavenumber.  The garbled log10(1/Gamma) term is read as the number
    of digits.  Pinned by the nine direction counts the paper prints.
"""
from __future__ import annotations

import numpy as np


def box_radius(a: float) -> float:
    """Radius of the sphere enclosing a cubic box of edge a (Sec. II.A, R^s)."""
    return a * np.sqrt(3.0) / 2.0


def multipole_count(k: complex, a: float, digits: float) -> int:
    """Number of multipoles L from the excess-bandwidth formula (Sec. II.A)."""
    x = 2.0 * abs(k) * box_radius(a)
    return int(np.floor(x + 1.8 * x ** (1.0 / 3.0) * digits ** (2.0 / 3.0)))


def gauss_legendre(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre nodes (ascending) and weights on [-1, 1].

    Golub-Welsch: the nodes are the eigenvalues of the symmetric tridiagonal
    Jacobi matrix of the Legendre three-term recurrence, with off-diagonal
    beta_i = i / sqrt(4 i^2 - 1); the weights are 2 * (first eigenvector
    component)^2.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    i = np.arange(1, n, dtype=np.float64)
    beta = i / np.sqrt(4.0 * i * i - 1.0)
    J = np.diag(beta, 1) + np.diag(beta, -1)
    nodes, vecs = np.linalg.eigh(J)
    weights = 2.0 * vecs[0, :] ** 2
    order = np.argsort(nodes)
    return nodes[order], weights[order]


def nphi_for(L: int, rule: str = "benchmark") -> int:
    if rule == "benchmark":
        return 2 * (L + 1)
    if rule == "paper":
        return 2 * L + 1
    raise ValueError(f"unknown nphi rule {rule!r}")


def direction_grid(L: int, rule: str = "benchmark"):
    """Unit directions k_p (N_dir x 3) and quadrature weights w_p (Sec. II.A, Eq. 6).

    Weights integrate over the unit sphere: sum_p w_p = 4 pi.
    """
    x, wx = gauss_legendre(L + 1)
    nphi = nphi_for(L, rule)
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    sin_t = np.sqrt(np.clip(1.0 - x * x, 0.0, None))
    kx = (sin_t[:, None] * np.cos(phi)[None, :]).ravel()
    ky = (sin_t[:, None] * np.sin(phi)[None, :]).ravel()
    kz = np.repeat(x, nphi)
    khat = np.stack([kx, ky, kz], axis=1)
    w = np.repeat(wx, nphi) * (2.0 * np.pi / nphi)
    return khat, w
