"""Pins for the oracle's storage count and memory saving (Sec. III).

The memory saving the paper reports is 1 - (stored elements) / (elements of
the uncompressed operators).  What each format stores is fixed by its
restoration formula:
  * Tucker-3D, Eq. 9, per direction p: the core r1 r2 r3 and the three
    factors n_i r_i;
  * TT-3D, Eq. 13, per direction: U1 (n1 r1), the middle core r1 n2 r2 and
    the last factor n3 r2;
  * Tucker-4D, Eq. 11: one core r1 r2 r3 r4 and four factors n_i r_i, the
    fourth over the directions;
  * H-Tucker, Eq. 12 and Fig. 3(c): four leaf bases n_i r_i, the two
    transfer tensors r1 r2 r12 and r3 r4 r34 and the root matrix r12 r34;
  * TT-4D, Eq. 14: U1 (n1 r1), two middle cores r1 n2 r2 and r2 n3 r3, and
    the direction factor n_dir r3.
Each count below is written out from those formulas for tensors built with
known ranks (which the decompositions recover exactly at a tiny tolerance),
so dropping or double-counting any one stored array fails a test.
"""
import numpy as np
import pytest

from oracle import decomp as D
from oracle import pipeline as pl


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _orth(rng, n, r):
    return np.linalg.qr(_crandn(rng, n, r))[0]


def _tucker_tensor(rng, n, r):
    T = _crandn(rng, *r)
    for i in range(len(n)):
        T = D.mode_product(T, _orth(rng, n[i], r[i]), i)
    return T


N3D = (9, 8, 10)


def test_uncompressed_store_counts_every_element():
    rng = np.random.default_rng(20)
    ops = [_crandn(rng, *N3D) for _ in range(3)]
    comp = pl.compress(ops, "4d", "none", 0.0)
    assert comp.elements() == 9 * 8 * 10 * 3
    assert comp.saving() == 0.0


def test_tucker3d_storage():
    rng = np.random.default_rng(21)
    ranks = [(3, 2, 4), (2, 5, 3), (4, 4, 1)]
    ops = [_tucker_tensor(rng, N3D, r) for r in ranks]
    comp = pl.compress(ops, "3d", "tucker", 1e-11)
    assert [t.ranks for t in comp.parts] == ranks
    n1, n2, n3 = N3D
    want = sum(r1 * r2 * r3 + n1 * r1 + n2 * r2 + n3 * r3 for r1, r2, r3 in ranks)
    assert comp.elements() == want
    assert comp.saving() == pytest.approx(1.0 - want / (n1 * n2 * n3 * 3), abs=1e-15)


def test_tt3d_storage():
    rng = np.random.default_rng(22)
    n1, n2, n3 = N3D
    ranks = [(3, 4), (2, 2), (5, 3)]
    ops = [np.einsum("ai,ibj,cj->abc", _crandn(rng, n1, r1), _crandn(rng, r1, n2, r2), _crandn(rng, n3, r2))
           for r1, r2 in ranks]
    comp = pl.compress(ops, "3d", "tt", 1e-11)
    assert [t.ranks for t in comp.parts] == ranks
    want = sum(n1 * r1 + r1 * n2 * r2 + n3 * r2 for r1, r2 in ranks)
    assert comp.elements() == want
    assert comp.saving() == pytest.approx(1.0 - want / (n1 * n2 * n3 * 3), abs=1e-15)


def test_tucker4d_storage():
    rng = np.random.default_rng(23)
    n = N3D + (11,)
    r = (3, 2, 4, 5)
    T = _tucker_tensor(rng, n, r)
    comp = pl.compress([T[..., p] for p in range(n[3])], "4d", "tucker", 1e-11)
    assert comp.parts.ranks == r
    want = r[0] * r[1] * r[2] * r[3] + sum(ni * ri for ni, ri in zip(n, r))
    assert comp.elements() == want
    assert comp.saving() == pytest.approx(1.0 - want / np.prod(n), abs=1e-15)


def test_htucker_storage():
    rng = np.random.default_rng(24)
    n = N3D + (11,)
    r, r12, r34 = (3, 2, 4, 3), 4, 4
    C12 = np.linalg.qr(_crandn(rng, r[0] * r[1], r12))[0].reshape(r[0], r[1], r12)
    C34 = np.linalg.qr(_crandn(rng, r[2] * r[3], r34))[0].reshape(r[2], r[3], r34)
    T = np.einsum("ijs,st,klt->ijkl", C12, _crandn(rng, r12, r34), C34)
    for i in range(4):
        T = D.mode_product(T, _orth(rng, n[i], r[i]), i)
    comp = pl.compress([T[..., p] for p in range(n[3])], "4d", "htucker", 1e-11)
    assert comp.parts.ranks == r + (r12, r34)
    want = (sum(ni * ri for ni, ri in zip(n, r)) + r[0] * r[1] * r12 + r[2] * r[3] * r34 + r12 * r34)
    assert comp.elements() == want
    assert comp.saving() == pytest.approx(1.0 - want / np.prod(n), abs=1e-15)


def test_tt4d_storage():
    rng = np.random.default_rng(25)
    n1, n2, n3, n4 = N3D + (11,)
    r1, r2, r3 = 3, 4, 2
    T = np.einsum("ai,ibj,jck,pk->abcp", _crandn(rng, n1, r1), _crandn(rng, r1, n2, r2),
                  _crandn(rng, r2, n3, r3), _crandn(rng, n4, r3))
    comp = pl.compress([T[..., p] for p in range(n4)], "4d", "tt", 1e-11)
    assert comp.parts.ranks == (r1, r2, r3)
    want = n1 * r1 + r1 * n2 * r2 + r2 * n3 * r3 + n4 * r3
    assert comp.elements() == want
    assert comp.saving() == pytest.approx(1.0 - want / (n1 * n2 * n3 * n4), abs=1e-15)
