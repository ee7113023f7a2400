"""Pins for the decompositions (Algs. 1-3) and restorations (Figs. 3, 4).

* exact recovery of tensors built with a known multilinear / TT / H-Tucker rank;
* the truncation error bounds the algorithms guarantee
  (HOSVD: ||T - T^||^2 <= sum of discarded sigma^2 over the modes, and at least
  the largest single-mode discarded energy by Eckart-Young; TT-SVD: <= sum of the
  per-step discarded energies; every rule: <= gamma ||T||);
* the matrix-step restorations of Figs. 3 and 4 agree with brute-force loops.
"""
import numpy as np
import pytest

from oracle import decomp as D
from oracle import pipeline as pl
from seeded_inputs import field_spectra


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _orth(rng, n, r):
    q, _ = np.linalg.qr(_crandn(rng, n, r))
    return q


def test_truncation_rank_rule():
    s = np.array([3.0, 2.0, 1.0, 0.5])
    assert D.truncation_rank(s, np.sqrt(1.25)) == 2
    assert D.truncation_rank(s, 1.1) == 3
    assert D.truncation_rank(s, 0.0) == 4
    assert D.truncation_rank(s, 100.0) == 1
    assert D.truncation_rank(s, 0.4, "paper_sv") == 2


def test_mode_product_definition():
    rng = np.random.default_rng(0)
    X = _crandn(rng, 2, 3, 4)
    M = _crandn(rng, 5, 3)
    Y = D.mode_product(X, M, 1)
    ref = np.zeros((2, 5, 4), complex)
    for a in range(2):
        for j in range(5):
            for c in range(4):
                ref[a, j, c] = sum(X[a, k, c] * M[j, k] for k in range(3))
    np.testing.assert_allclose(Y, ref, atol=1e-13)


def test_tucker_recovers_known_multilinear_rank():
    rng = np.random.default_rng(1)
    n, r = (9, 8, 10, 7), (3, 4, 2, 5)
    C = _crandn(rng, *r)
    T = C
    for i in range(4):
        T = D.mode_product(T, _orth(rng, n[i], r[i]), i)
    tk = D.tucker_hosvd(T, 1e-10)
    assert tk.ranks == r
    np.testing.assert_allclose(D.tucker_restore(tk), T, atol=1e-12 * np.abs(T).max())
    for U in tk.factors:
        np.testing.assert_allclose(U.conj().T @ U, np.eye(U.shape[1]), atol=1e-13)


def test_tt_recovers_known_tt_rank():
    rng = np.random.default_rng(2)
    n1, n2, n3, n4 = 6, 7, 5, 8
    U1, C1, C2, U4 = _crandn(rng, n1, 3), _crandn(rng, 3, n2, 4), _crandn(rng, 4, n3, 2), _crandn(rng, n4, 2)
    T = np.einsum("ai,ibj,jck,pk->abcp", U1, C1, C2, U4)
    tt = D.tt_svd(T, 1e-11)
    assert tt.ranks == (3, 4, 2)
    np.testing.assert_allclose(D.tt_restore(tt), T, atol=1e-11 * np.abs(T).max())
    T3 = np.einsum("ai,ibj,cj->abc", U1, C1, _crandn(rng, n3, 4))
    tt3 = D.tt_svd(T3, 1e-11)
    assert tt3.ranks == (3, 4)
    np.testing.assert_allclose(D.tt_restore(tt3), T3, atol=1e-11 * np.abs(T3).max())


def test_htucker_recovers_known_hierarchical_rank():
    rng = np.random.default_rng(3)
    n, r = (8, 7, 9, 10), (3, 2, 4, 3)
    r12, r34 = 4, 4  # W12 = C12 B C34^T has rank min(r12, r34)
    C12 = np.linalg.qr(_crandn(rng, r[0] * r[1], r12))[0].reshape(r[0], r[1], r12)
    C34 = np.linalg.qr(_crandn(rng, r[2] * r[3], r34))[0].reshape(r[2], r[3], r34)
    B = _crandn(rng, r12, r34)
    W = np.einsum("ijs,st,klt->ijkl", C12, B, C34)
    T = W
    for i in range(4):
        T = D.mode_product(T, _orth(rng, n[i], r[i]), i)
    ht = D.htucker_svd(T, 1e-11)
    assert ht.ranks == r + (r12, r34)
    np.testing.assert_allclose(D.htucker_restore(ht), T, atol=1e-11 * np.abs(T).max())


@pytest.fixture(scope="module")
def small_ops():
    plan = pl.Plan(K=(4, 4, 4), L=3)
    return plan, pl.operators(plan)


@pytest.mark.parametrize("gamma", [1e-2, 1e-3, 1e-5])
def test_hosvd_error_bounds(small_ops, gamma):
    _, ops = small_ops
    for T in ops[::7]:
        tk = D.tucker_hosvd(T, gamma)
        err = np.linalg.norm(D.tucker_restore(tk) - T)
        disc = [np.sum(s[r:] ** 2) for s, r in zip(tk.sigmas, tk.ranks)]
        assert err ** 2 <= sum(disc) * (1 + 1e-9) + 1e-24
        assert err >= np.sqrt(max(disc)) * (1 - 1e-9)
        assert err <= gamma * np.linalg.norm(T) * (1 + 1e-12)


@pytest.mark.parametrize("gamma", [1e-2, 1e-4])
def test_tt_error_bounds(small_ops, gamma):
    _, ops = small_ops
    T4 = pl.stack4d(ops)
    for T in (ops[3], T4):
        tt = D.tt_svd(T, gamma)
        err = np.linalg.norm(D.tt_restore(tt) - T)
        disc = sum(np.sum(s[r:] ** 2) for s, r in zip(tt.sigmas, tt.ranks))
        assert err ** 2 <= disc * (1 + 1e-9) + 1e-24
        assert err <= gamma * np.linalg.norm(T) * (1 + 1e-12)


@pytest.mark.parametrize("gamma", [1e-2, 1e-4])
def test_htucker_and_tucker4d_error_bounds(small_ops, gamma):
    _, ops = small_ops
    T4 = pl.stack4d(ops)
    ht = D.htucker_svd(T4, gamma)
    assert np.linalg.norm(D.htucker_restore(ht) - T4) <= gamma * np.linalg.norm(T4) * (1 + 1e-12)
    tk = D.tucker_hosvd(T4, gamma)
    assert np.linalg.norm(D.tucker_restore(tk) - T4) <= gamma * np.linalg.norm(T4) * (1 + 1e-12)


def test_full_rank_reproduces_operator(small_ops):
    _, ops = small_ops
    T = ops[2]
    np.testing.assert_allclose(D.tucker_restore(D.tucker_hosvd(T, 0.0)), T, atol=1e-12 * np.abs(T).max())
    np.testing.assert_allclose(D.tt_restore(D.tt_svd(T, 0.0)), T, atol=1e-12 * np.abs(T).max())


def test_restoration_steps_match_brute_force():
    rng = np.random.default_rng(4)
    n, r = (3, 4, 5), (2, 3, 2)
    C = _crandn(rng, *r)
    U = [_crandn(rng, n[i], r[i]) for i in range(3)]
    ref = np.zeros(n, complex)
    for i in range(n[0]):
        for j in range(n[1]):
            for k in range(n[2]):
                ref[i, j, k] = sum(C[a, b, c] * U[0][i, a] * U[1][j, b] * U[2][k, c]
                                   for a in range(r[0]) for b in range(r[1]) for c in range(r[2]))
    np.testing.assert_allclose(D.tucker3d_restore_steps(C, *U), ref, atol=1e-12)
    # TT-3D, Fig. 4(a)
    U1, C1, U3 = _crandn(rng, 3, 2), _crandn(rng, 2, 4, 3), _crandn(rng, 5, 3)
    ref = np.zeros(n, complex)
    for i in range(3):
        for j in range(4):
            for k in range(5):
                ref[i, j, k] = sum(U1[i, a] * C1[a, j, b] * U3[k, b] for a in range(2) for b in range(3))
    np.testing.assert_allclose(D.tt3d_restore_steps(U1, C1, U3), ref, atol=1e-12)


def test_4d_per_direction_restorations(small_ops):
    _, ops = small_ops
    T4 = pl.stack4d(ops)
    for decomp in ("tucker", "tt", "htucker"):
        comp = pl.compress(ops, "4d", decomp, 1e-3)
        full = {"tucker": lambda: D.tucker_restore(comp.parts),
                "tt": lambda: D.tt_restore(comp.parts),
                "htucker": lambda: D.htucker_restore(comp.parts)}[decomp]()
        for p in (0, 5, len(ops) - 1):
            np.testing.assert_allclose(comp.restore(p), full[..., p], atol=1e-12 * np.abs(T4).max())
        assert 0.0 < comp.saving() < 1.0


@pytest.mark.parametrize("fmt,decomp", [("3d", "tucker"), ("3d", "tt"), ("4d", "tucker"),
                                        ("4d", "tt"), ("4d", "htucker")])
def test_compressed_translation_error_tracks_tolerance(small_ops, fmt, decomp):
    plan, ops = small_ops
    gamma = 1e-3
    S = field_spectra(7, plan.n_dir, 1, plan.K)
    dirs = [0, 9, 17, 30]
    ref = pl.translate_with(lambda p: ops[p], S, dirs)
    comp = pl.compress(ops, fmt, decomp, gamma)
    out = pl.translate_with(comp.restore, S, dirs)
    err = pl.relative_l2(out[dirs], ref[dirs])
    assert err <= 2.0 * gamma
    # "none" reproduces the plain store exactly
    none = pl.compress(ops, "none", "none", 0.0)
    assert np.array_equal(pl.translate_with(none.restore, S, dirs)[dirs], ref[dirs])
