"""Pins for the far-field steps around the translation (Eqs. 4 and 6).

* physics: with point-source patterns P^+(k, b_n) = (alpha_n, beta_n)
  e^{+jk k.(r_n - r_v)} (Eq. 3 for a point source), aggregation, the
  translation of Eq. 5 and disaggregation together give, times -jk/(4 pi),
  the Green's-function sum over every pair of points in far boxes,
  sum_n (conj(alpha_m) alpha_n + conj(beta_m) beta_n) e^{-jk R_mn}/R_mn I_n,
  to the accuracy of the multipole count (Sec. II.A);
* adjoint identity: sum_m conj(I_m) y_m = sum_p w_p sum conj(A_p) B_p for
  y = disaggregate(P, w, B), A = aggregate(P, I), which a dropped or misplaced
  conjugate, weight or index breaks.
"""
import numpy as np
import pytest

from oracle import directions as dr
from oracle import farfield as ff
from oracle import operator as op
from oracle import pipeline as pl
from oracle import translate as tr
from seeded_inputs import complex_gaussian, uniform01


def _point_sources(seed, K, nb, a):
    """Positions r_n (inside their boxes), box indices and box centres."""
    V = K[0] * K[1] * K[2]
    u = uniform01(seed, np.arange(3 * nb * V, dtype=np.uint64)).reshape(nb, K[2], K[1], K[0], 3)
    z, y, x = np.meshgrid(np.arange(K[2]), np.arange(K[1]), np.arange(K[0]), indexing="ij")
    centre = np.stack([x, y, z], axis=-1) * a                       # (Kz, Ky, Kx, 3)
    pos = centre[None] + (u - 0.5) * a                              # (nb, Kz, Ky, Kx, 3)
    return pos, centre


@pytest.mark.parametrize("K,nb,digits", [((5, 4, 6), 2, 5), ((6, 5, 5), 1, 6)])
def test_far_field_matvec_reproduces_green_function(K, nb, digits):
    a, k = 0.5, 2 * np.pi
    L = dr.multipole_count(k, a, digits)
    plan = pl.Plan(K=K, a=a, k0=k, L=L, nphi_rule="paper", near_rule="kappa")
    kh, w = dr.direction_grid(L, "paper")
    pos, centre = _point_sources(17, K, nb, a)
    rho = pos - centre[None]
    ab = complex_gaussian(18, 2 * nb * K[0] * K[1] * K[2]).reshape(2, nb, K[2], K[1], K[0])
    phase = np.exp(1j * k * np.einsum("pd,izyxd->pizyx", kh, rho))
    P = np.stack([ab[0][None] * phase, ab[1][None] * phase], axis=1)  # (p, c, i, z, y, x)
    I = complex_gaussian(19, nb * K[0] * K[1] * K[2]).reshape(1, nb, K[2], K[1], K[0])

    A = ff.aggregate(P, I)
    B = tr.translate_fft(pl.operators(plan), A)
    y = (-1j * k / (4 * np.pi)) * ff.disaggregate(P, w, B)

    # direct sum over point pairs in far boxes (near rule of the plan)
    box = np.stack(np.meshgrid(np.arange(K[2]), np.arange(K[1]), np.arange(K[0]), indexing="ij"), -1)
    bx = np.broadcast_to(box[None], (nb,) + box.shape).reshape(-1, 3)[:, ::-1]   # (x, y, z)
    r = pos.reshape(-1, 3)
    al, be, cur = ab[0].ravel(), ab[1].ravel(), I[0].ravel()
    d = bx[:, None, :] - bx[None, :, :]
    far = ~op.near_mask(d[..., 0], d[..., 1], d[..., 2], "kappa")
    R = np.linalg.norm(r[:, None, :] - r[None, :, :], axis=-1)
    G = np.where(far, np.exp(-1j * k * R) / np.where(far, R, 1.0), 0.0)
    coup = np.conj(al)[:, None] * al[None, :] + np.conj(be)[:, None] * be[None, :]
    ref = (coup * G) @ cur
    assert np.count_nonzero(far) > 0
    err = np.linalg.norm(y[0].ravel() - ref) / np.linalg.norm(ref)
    assert err < 10.0 ** (-digits), err


def test_dropping_the_conjugate_breaks_the_matvec():
    # P^- = P^+ (no conjugate) in Eq. 6 no longer gives the Green's function
    K, nb, a, k = (5, 4, 6), 1, 0.5, 2 * np.pi
    L = dr.multipole_count(k, a, 5)
    plan = pl.Plan(K=K, a=a, k0=k, L=L, nphi_rule="paper", near_rule="kappa")
    kh, w = dr.direction_grid(L, "paper")
    pos, centre = _point_sources(21, K, nb, a)
    phase = np.exp(1j * k * np.einsum("pd,izyxd->pizyx", kh, pos - centre[None]))
    P = np.stack([phase, 0 * phase], axis=1)
    I = complex_gaussian(22, nb * K[0] * K[1] * K[2]).reshape(1, nb, K[2], K[1], K[0])
    B = tr.translate_fft(pl.operators(plan), ff.aggregate(P, I))
    good = ff.disaggregate(P, w, B)
    bad = np.einsum("p,pcizyx,pcrzyx->rizyx", w, P, B)
    assert np.linalg.norm(bad - good) > 0.5 * np.linalg.norm(good)


def test_adjoint_identity():
    rng_shape = (7, 2, 3, 2, 3, 4)     # (p, c, i, z, y, x)
    P = complex_gaussian(31, int(np.prod(rng_shape))).reshape(rng_shape)
    I = complex_gaussian(32, 2 * 3 * 2 * 3 * 4).reshape(2, 3, 2, 3, 4)
    B = complex_gaussian(33, 7 * 2 * 2 * 2 * 3 * 4).reshape(7, 2, 2, 2, 3, 4)
    w = np.linspace(0.3, 1.7, 7)
    y = ff.disaggregate(P, w, B)
    A = ff.aggregate(P, I)
    lhs = np.vdot(I, y)
    rhs = np.sum(w[:, None] * np.einsum("pcrzyx,pcrzyx->pc", np.conj(A), B))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
