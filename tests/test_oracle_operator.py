"""Pins for the translation operator (Eq. 7), its embedding and the translation (Eq. 5).

* Gegenbauer / plane-wave expansion: the quadrature of e^{-jk k.d} T_L(k, X)
  over the direction grid reproduces the free-space Green's function
  e^{-jk|X+d|}/|X+d| (this fixes the l = 0 term, the (-j)^l phase and the
  Hankel kind of Eq. 7);
* symmetry: T depends only on k.R^ and |R|, so it is unchanged by any signed
  axis permutation applied to both k and R, and by k -> -k, R -> -R, and two
  offsets of equal length that no lattice symmetry relates (Pythagorean
  quadruples such as (3, 4, 0) and (5, 0, 0)) give equal values for directions
  at equal angles to them;
* near offsets are zero;
* the FFT route of Eq. 5 equals the brute-force Toeplitz sum.
"""
import itertools

import numpy as np
import pytest

from oracle import directions as dr
from oracle import operator as op
from oracle import pipeline as pl
from oracle import translate as tr
from oracle.special import legendre_all, spherical_hankel2_all


def _T_point(khat, X, k, L):
    R = np.linalg.norm(X)
    h = spherical_hankel2_all(L, np.array([k * R]))[:, 0]
    P = legendre_all(L, np.asarray(khat) @ (X / R))
    l = np.arange(L + 1)
    return ((-1j) ** l * (2 * l + 1) * h) @ P


@pytest.mark.parametrize("X,d", [((1.0, 1.5, 0.5), (0.1, -0.15, 0.2)),
                                 ((2.0, 0.0, 0.0), (0.0, 0.25, -0.2)),
                                 ((0.0, -1.5, 1.5), (0.2, 0.2, 0.2))])
def test_plane_wave_expansion_reproduces_green_function(X, d):
    k = 2 * np.pi
    L = 16
    kh, w = dr.direction_grid(L, "paper")
    X, d = np.array(X), np.array(d)
    # operator_at takes integer offsets scaled by a: use a = 1 and X itself
    T = np.array([_T_point(kh[p], X, k, L) for p in range(len(kh))])
    # the same values through operator_at (X on an a = 0.5 grid)
    Xi = (X / 0.5).round().astype(int)
    T2 = np.array([op.operator_at(kh[p], Xi[0], Xi[1], Xi[2], 0.5, k, L, near_rule="kappa", kappa=0.0)
                   for p in range(len(kh))])
    np.testing.assert_allclose(T2, T, rtol=1e-11)
    q = (-1j * k / (4 * np.pi)) * np.sum(w * np.exp(-1j * k * (kh @ d)) * T)
    R = np.linalg.norm(X + d)
    np.testing.assert_allclose(q, np.exp(-1j * k * R) / R, rtol=1e-8)


@pytest.mark.parametrize("eps_r,rtol", [(2 - 1j, 1e-8), (2 - 2j, 1e-8), (2 - 8j, 1e-6)])
def test_plane_wave_expansion_in_a_lossy_medium(eps_r, rtol):
    """Sec. III.A.5: with the complex wavenumber k = k0 sqrt(eps_r) the same
    quadrature reproduces the lossy Green's function e^{-jk|X+d|}/|X+d|, which
    fixes the branch of sqrt(eps_r) (decay for Im eps_r < 0) and the complex
    Hankel function."""
    k0 = 2 * np.pi
    k = op.medium_wavenumber(k0, eps_r)
    assert k.imag < 0
    X, d = np.array([1.0, 1.5, 0.5]), np.array([0.1, -0.15, 0.2])
    L = 24
    kh, w = dr.direction_grid(L, "paper")
    Xi = (X / 0.5).round().astype(int)
    T = np.array([op.operator_at(kh[p], Xi[0], Xi[1], Xi[2], 0.5, k0, L, near_rule="kappa", kappa=0.0,
                                 eps_r=eps_r) for p in range(len(kh))])
    q = (-1j * k / (4 * np.pi)) * np.sum(w * np.exp(-1j * k * (kh @ d)) * T)
    R = np.linalg.norm(X + d)
    ref = np.exp(-1j * k * R) / R
    assert abs(q - ref) <= rtol * abs(ref)


def test_paper_prefactor_in_a_medium():
    # c = -k^2 eta / (16 pi^2) with k = k0 sqrt(eps_r), eta = eta0 / sqrt(eps_r)
    for eps in (1.0, 2.0, 2 - 8j):
        c = op.prefactor_value(2 * np.pi, "paper", eps)
        ref = -(2 * np.pi) ** 2 * np.sqrt(complex(eps)) * op.ETA0 / (16 * np.pi ** 2)
        assert abs(c - ref) <= 1e-14 * abs(ref)


def test_direction_mode_rank_is_spherical_harmonic_count():
    """As a function of k_p, T_p is a polynomial of degree L in k_p (the Legendre
    terms P_l(k_p . R^), l = 0..L), so the direction-mode unfolding of T_4D has
    rank (L+1)^2, the number of spherical harmonics of degree <= L.  Table II
    prints r4 = r3 = 225 = 15^2 for L = 14; a sum starting at l = 1 (the printed
    lower limit of Eq. 7) would give (L+1)^2 - 1."""
    L, K = 5, (4, 4, 4)
    plan = pl.Plan(K=K, L=L, nphi_rule="paper", near_rule="kappa")
    T4 = pl.stack4d(pl.operators(plan))
    s = np.linalg.svd(T4.reshape(-1, plan.n_dir), compute_uv=False)
    assert plan.n_dir > (L + 1) ** 2
    assert int(np.sum(s > 1e-10 * s[0])) == (L + 1) ** 2
    # the l = 0 term removed: one harmonic fewer
    kh = plan.directions()
    ax = op.offset_axes(K)
    dx, dy, dz = np.meshgrid(*ax, indexing="ij")
    d = np.sqrt(dx * dx + dy * dy + dz * dz)
    far = ~op.near_mask(dx, dy, dz, "kappa")
    h0 = np.zeros(d.shape, dtype=np.complex128)
    h0[far] = spherical_hankel2_all(0, plan.k0 * plan.a * d[far])[0]
    cols = []
    for p in range(plan.n_dir):
        T = op.operator_grid(kh[p], K, plan.a, plan.k0, L, "kappa") - h0
        cols.append(np.fft.fftn(op.embed(T, K, plan.n)).ravel())
    s1 = np.linalg.svd(np.stack(cols, axis=1), compute_uv=False)
    assert int(np.sum(s1 > 1e-10 * s1[0])) == (L + 1) ** 2 - 1


def test_dropping_monopole_breaks_expansion():
    # a summation from l = 1 (the printed lower limit) misses the Green's function
    k, L = 2 * np.pi, 16
    kh, w = dr.direction_grid(L, "paper")
    X, d = np.array([1.0, 1.5, 0.5]), np.array([0.1, -0.15, 0.2])
    T = np.array([_T_point(kh[p], X, k, L) for p in range(len(kh))])
    h0 = spherical_hankel2_all(0, np.array([k * np.linalg.norm(X)]))[0, 0]
    q = (-1j * k / (4 * np.pi)) * np.sum(w * np.exp(-1j * k * (kh @ d)) * (T - h0))
    R = np.linalg.norm(X + d)
    assert abs(q - np.exp(-1j * k * R) / R) > 1e-2


def _signed_perms():
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            M = np.zeros((3, 3), dtype=int)
            for i, j in enumerate(perm):
                M[i, j] = signs[i]
            yield M


def test_operator_symmetries():
    K = (4, 3, 5)
    kh, _ = dr.direction_grid(4)
    rng = np.random.default_rng(3)
    ax = op.offset_axes((6, 6, 6))
    dx, dy, dz = np.meshgrid(*ax, indexing="ij")
    for p in rng.choice(len(kh), 4, replace=False):
        base = op.operator_at(kh[p], dx, dy, dz, 0.5, 2 * np.pi, 4)
        for M in list(_signed_perms())[::5]:
            k2 = M @ kh[p]
            D = np.einsum("ij,jxyz->ixyz", M, np.stack([dx, dy, dz]))
            rot = op.operator_at(k2, D[0], D[1], D[2], 0.5, 2 * np.pi, 4)
            np.testing.assert_allclose(rot, base, rtol=1e-12, atol=1e-14)
        anti = op.operator_at(-kh[p], -dx, -dy, -dz, 0.5, 2 * np.pi, 4)
        np.testing.assert_allclose(anti, base, rtol=1e-12, atol=1e-14)
    del K


# offsets of equal length not related by a signed axis permutation
_EQUAL_LENGTH = [[(3, 4, 0), (5, 0, 0), (0, -3, 4)],
                 [(1, 2, 2), (3, 0, 0), (2, -1, -2)],
                 [(2, 3, 6), (7, 0, 0), (6, -2, 3)],
                 [(1, 4, 8), (4, 4, 7), (9, 0, 0)]]


@pytest.mark.parametrize("group", _EQUAL_LENGTH)
def test_operator_depends_only_on_angle_and_distance(group):
    """Eq. 7 is a function of k.R^ and |R| alone: for each offset of the group
    a direction at the same angle to it (rotated about no lattice axis) gives
    the same value as the first offset with a random direction."""
    rng = np.random.default_rng(sum(map(sum, group)))
    a, k0, L = 0.5, 2 * np.pi, 6
    for _ in range(3):
        k1 = rng.normal(size=3)
        k1 /= np.linalg.norm(k1)
        d1 = np.array(group[0], dtype=float)
        c = k1 @ d1 / np.linalg.norm(d1)
        ref = op.operator_at(k1, *group[0], a, k0, L)
        assert abs(ref) > 0
        for d in group[1:]:
            u = np.array(d, dtype=float) / np.linalg.norm(d)
            e = rng.normal(size=3)
            e -= (e @ u) * u
            e /= np.linalg.norm(e)
            k2 = c * u + np.sqrt(max(0.0, 1 - c * c)) * e
            np.testing.assert_allclose(op.operator_at(k2, *d, a, k0, L), ref, rtol=1e-11)
        # a different angle to the same offset changes the value
        k3 = -c * d1 / np.linalg.norm(d1) + np.sqrt(max(0.0, 1 - c * c)) * np.cross(k1, d1) / \
            max(np.linalg.norm(np.cross(k1, d1)), 1e-300)
        if abs(c) > 0.1:
            assert abs(op.operator_at(k3, *group[0], a, k0, L) - ref) > 1e-6 * abs(ref)


def test_near_offsets_are_zero_and_far_are_not():
    kh, _ = dr.direction_grid(3)
    T = op.operator_grid(kh[5], (4, 4, 4), 0.5, 2 * np.pi, 3)
    c = 3  # index of offset 0
    assert np.all(T[c - 1:c + 2, c - 1:c + 2, c - 1:c + 2] == 0)
    far = np.ones(T.shape, bool)
    far[c - 1:c + 2, c - 1:c + 2, c - 1:c + 2] = False
    assert np.all(np.abs(T[far]) > 0)
    Tk = op.operator_grid(kh[5], (4, 4, 4), 0.5, 2 * np.pi, 3, near_rule="kappa")
    # kappa rule: |Delta|^2 < 12 is near, so (2,2,1) (|.|^2 = 9) is near, (3,2,0) (13) is far
    assert Tk[c + 2, c + 2, c + 1] == 0 and Tk[c + 3, c + 2, c] != 0


def test_embedding_places_offsets_circularly():
    K, n = (3, 2, 4), (6, 4, 8)
    g = np.arange(5 * 3 * 7).reshape(5, 3, 7) + 1.0
    E = op.embed(g, K, n)
    for ix, dx in enumerate(range(-2, 3)):
        for iy, dy in enumerate(range(-1, 2)):
            for iz, dz in enumerate(range(-3, 4)):
                assert E[dx % 6, dy % 4, dz % 8] == g[ix, iy, iz]
    assert np.all(E[3, :, :] == 0) and np.all(E[:, 2, :] == 0) and np.all(E[:, :, 4] == 0)


@pytest.mark.parametrize("K", [(3, 3, 3), (3, 4, 5), (5, 2, 6), (4, 4, 4)])
def test_fft_translation_equals_direct_sum(K):
    plan = pl.Plan(K=K, L=3)
    kh = plan.directions()
    rng = np.random.default_rng(sum(K))
    for p in (0, len(kh) // 3):
        Tg = op.operator_grid(kh[p], K, plan.a, plan.k0, plan.L)
        Th = op.fft_operator(kh[p], K, plan.n, plan.a, plan.k0, plan.L)
        A = rng.standard_normal(K[::-1]) + 1j * rng.standard_normal(K[::-1])
        Bf = tr.translate_field_fft(Th, A)
        Bd = tr.translate_field_direct(Tg, A)
        np.testing.assert_allclose(Bf, Bd, rtol=0, atol=1e-12 * np.abs(Bd).max())
        # one output box through the pointwise direct sum
        v = (K[0] - 1, 0, K[2] // 2)
        f = lambda a, b, c: op.operator_at(kh[p], a, b, c, plan.a, plan.k0, plan.L)
        np.testing.assert_allclose(tr.translate_point_direct(f, A, v), Bd[v[2], v[1], v[0]],
                                   rtol=1e-10)


def test_embed_extent_rule():
    assert [pl.embed_extent(k) for k in (2, 3, 4, 5, 8, 12, 17, 32, 33, 64, 128)] == \
        [4, 8, 8, 16, 16, 32, 64, 64, 128, 128, 256]
