"""Pins for the oracle's special functions and direction grid (Sec. II.A, Eq. 7).

Each check compares against something other than the oracle's own formula:
library routines (scipy/numpy), closed forms, or numbers printed in the paper.
"""
import os

import numpy as np
import pytest
import scipy.special as sp

from oracle import directions as dr
from oracle import special as sf

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("x", [np.array([0.05, 0.3, 1.0, 3.14159, 6.28, 17.7, 45.0, 120.0])])
def test_hankel2_matches_scipy(x):
    lmax = 25
    H = sf.spherical_hankel2_all(lmax, x)
    for l in range(lmax + 1):
        ref = sp.spherical_jn(l, x) - 1j * sp.spherical_yn(l, x)
        np.testing.assert_allclose(H[l], ref, rtol=1e-12, atol=0)


def test_j_at_multiples_of_pi():
    # j_0 vanishes at m*pi; the downward recurrence must still give j_l there
    x = np.pi * np.arange(1, 12)
    J = sf.spherical_jn_all(10, x)
    for l in range(11):
        np.testing.assert_allclose(J[l], sp.spherical_jn(l, x), rtol=1e-10, atol=1e-15)


def test_hankel0_closed_form():
    x = np.linspace(0.1, 50, 97)
    h0 = sf.spherical_hankel2_all(0, x)[0]
    np.testing.assert_allclose(h0, 1j * np.exp(-1j * x) / x, rtol=1e-13)


def test_legendre_matches_scipy():
    t = np.linspace(-1, 1, 41)
    P = sf.legendre_all(30, t)
    for l in range(31):
        np.testing.assert_allclose(P[l], sp.eval_legendre(l, t), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 6, 9, 11, 15, 29])
def test_gauss_legendre_matches_numpy(n):
    x, w = dr.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=1e-14)
    np.testing.assert_allclose(w, wr, atol=1e-14)


@pytest.mark.parametrize("L", [2, 5, 8])
def test_direction_grid_quadrature(L):
    """The product rule integrates spherical polynomials of degree <= 2L+1 exactly
    (theta) and every trig polynomial of degree < N_phi (phi)."""
    kh, w = dr.direction_grid(L)
    np.testing.assert_allclose(np.linalg.norm(kh, axis=1), 1.0, atol=1e-14)
    assert kh.shape[0] == (L + 1) * 2 * (L + 1)
    np.testing.assert_allclose(w.sum(), 4 * np.pi, rtol=1e-14)
    # integral of z^2 over the sphere = 4 pi / 3; of x^2 y^2 = 4 pi / 15
    np.testing.assert_allclose(np.sum(w * kh[:, 2] ** 2), 4 * np.pi / 3, rtol=1e-13)
    np.testing.assert_allclose(np.sum(w * kh[:, 0] ** 2 * kh[:, 1] ** 2), 4 * np.pi / 15,
                               rtol=1e-12)
    # grid is closed under k -> -k (even N_phi, symmetric GL nodes)
    d = np.linalg.norm(kh[:, None, :] + kh[None, :, :], axis=2)
    assert np.all(d.min(axis=1) < 1e-12)


def _read_counts():
    path = os.path.join(os.path.dirname(__file__), "golden", "direction_counts.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows.append((float(parts[0]), float(parts[1]), complex(float(parts[2]), float(parts[3])),
                         int(parts[4])))
    return rows


@pytest.mark.parametrize("row", _read_counts())
def test_multipole_count_reproduces_printed_direction_counts(row):
    a, digits, eps_r, n_dir = row
    k = 2 * np.pi * np.sqrt(eps_r)
    L = dr.multipole_count(k, a, digits)
    assert (L + 1) * dr.nphi_for(L, "paper") == n_dir
