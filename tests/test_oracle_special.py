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


@pytest.mark.parametrize("lmax", [0, 1, 2, 3, 5])
def test_hankel2_small_order_matches_scipy(lmax):
    # few orders and moderate arguments: the downward recurrence grows little
    x = np.linspace(0.3, 40.0, 397)
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


# complex arguments of a lossy medium (Sec. III.A.5, Table IV): k = k0 sqrt(eps_r)
_LOSSY_Z = [2 * np.pi * np.sqrt(e) * 0.5 * r for e in (2 - 1j, 2 - 2j, 2 - 8j) for r in (2.0, 3.3, 9.0, 26.0)]


@pytest.mark.parametrize("z", _LOSSY_Z + [0.7 - 0.3j, 5.0 - 0.01j])
def test_hankel2_series_matches_high_precision_bessel(z):
    """The terminating series against h_l^(2) = sqrt(pi/2z) (J - iY)_{l+1/2}(z)
    evaluated by mpmath at 160 digits: J and Y are each of size e^{|Im z|} and
    cancel to e^{-|Im z|}, about 125 of those digits at Im z = -144."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 160
    lmax = 28
    H = sf.spherical_hankel2_all(lmax, np.array([z], dtype=np.complex128))[:, 0]
    zz = mp.mpc(z.real, z.imag)
    f = mp.sqrt(mp.pi / (2 * zz))
    half = mp.mpf(1) / 2
    for l in range(lmax + 1):
        ref = complex(f * (mp.besselj(l + half, zz) - 1j * mp.bessely(l + half, zz)))
        assert abs(H[l] - ref) <= 1e-10 * abs(ref), (l, H[l], ref)


def test_hankel2_series_on_the_real_axis_matches_scipy():
    x = np.array([0.4, 2.0, 7.5, 14.0, 30.0, 61.0])
    H = sf.spherical_hankel2_all(28, x.astype(np.complex128))
    for l in range(29):
        ref = sp.spherical_jn(l, x) - 1j * sp.spherical_yn(l, x)
        np.testing.assert_allclose(H[l], ref, rtol=1e-10, atol=0)


def test_hankel2_lossy_closed_forms():
    z = np.array(_LOSSY_Z)
    H = sf.spherical_hankel2_all(1, z)
    np.testing.assert_allclose(H[0], 1j * np.exp(-1j * z) / z, rtol=1e-13)
    np.testing.assert_allclose(H[1], np.exp(-1j * z) * (1j / z ** 2 - 1 / z), rtol=1e-13)
    # decays like e^{Im z} in a lossy medium
    assert np.all(np.abs(H[0]) <= np.exp(z.imag) / np.abs(z) * (1 + 1e-12))
