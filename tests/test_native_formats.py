"""Host-side checks of the library's compressed formats (no GPU needed).

fmmfft_compress_host runs the library's FP64 set-up for the plan's format
(Algs. 1-3) and restores every direction through the same restore schedule
the kernels follow (pre-pass products, then each direction's slab formula),
so these tests pin the decompositions and the descriptor plumbing of all five
formats against the oracle:
  * Tucker-3D, TT-3D, Tucker-4D, H-Tucker: the library's ranks equal the
    oracle's (same algorithm, same truncation rule), the restoration error
    equals the oracle's to rounding, and the stored element count and memory
    saving (Sec. III) equal the oracle's;
  * TT-4D: the library runs TT-SVD on the Tucker core of T_4D (budget
    gamma ||T|| / sqrt(7) per step); its error must stay within gamma and its
    ranks within the oracle's direct TT-SVD ranks at gamma / sqrt(7) * sqrt(3).
"""
import numpy as np
import pytest

from oracle import decomp as D
from oracle import pipeline as pl

TWO_PI = 2 * np.pi
FMT = {"3d": 3, "4d": 4}
DEC = {"tucker": 1, "tt": 2, "htucker": 3}


def _host(native, K, L, fmt, dec, tol, stats=False):
    h = native.fmmfft_plan_create(*K, 0.5, TWO_PI, L, FMT[fmt], DEC[dec], tol)
    try:
        ranks, R = native.fmmfft_compress_host(h)
        return (ranks, R, native.fmmfft_plan_stats(h)) if stats else (ranks, R)
    finally:
        native.fmmfft_plan_destroy(h)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fmt,dec,K,L,tol", [
    ("3d", "tucker", (6, 5, 7), 3, 1e-4),
    ("3d", "tt", (6, 5, 7), 3, 1e-4),
    ("3d", "tt", (8, 8, 8), 4, 1e-3),
    ("4d", "tucker", (6, 5, 7), 3, 1e-4),
    ("4d", "htucker", (6, 5, 7), 3, 1e-4),
    ("4d", "tucker", (8, 8, 8), 4, 1e-3),
    ("4d", "htucker", (8, 8, 8), 4, 1e-3),
    # y-z planes of 128 x 128 (the large-plane kernel's restore schedule)
    ("3d", "tucker", (3, 64, 64), 1, 1e-4),
    ("4d", "htucker", (3, 64, 64), 1, 1e-3),
])
def test_library_compression_matches_oracle(native, fmt, dec, K, L, tol):
    plan = pl.Plan(K=K, L=L)
    ops = pl.operators(plan)
    comp = pl.compress(ops, fmt, dec, tol)
    ranks, R, st = _host(native, K, L, fmt, dec, tol, stats=True)
    T4 = np.stack(ops)
    ref = np.stack([comp.restore(p) for p in range(plan.n_dir)])
    err, err_ref = _rel(R, T4), _rel(ref, T4)
    assert err <= tol
    assert abs(err - err_ref) <= 1e-9 + 1e-6 * err_ref
    if fmt == "3d":
        want = np.array([(list(t.ranks) + [0])[:3] for t in comp.parts])
        assert np.array_equal(ranks, want)
    else:
        got = [int(v) for v in ranks if v]
        assert tuple(got) == tuple(comp.parts.ranks)
    # equal ranks, so the stored element counts (Sec. III's memory saving,
    # counted by the oracle as the storage pins fix it) must agree exactly
    assert st["elements_compressed"] == comp.elements()
    assert st["elements_plain"] == int(np.prod(comp.shape))
    assert st["saving"] == pytest.approx(comp.saving(), abs=1e-12)


@pytest.mark.parametrize("K,L,tol", [((6, 5, 7), 3, 1e-4), ((8, 8, 8), 4, 1e-3)])
def test_library_tt4d_within_tolerance(native, K, L, tol):
    plan = pl.Plan(K=K, L=L)
    ops = pl.operators(plan)
    T4 = np.stack(ops)
    ranks, R, st = _host(native, K, L, "4d", "tt", tol, stats=True)
    assert _rel(R, T4) <= tol
    # its ranks are its own, so its element count is checked against Eq. 14's
    # storage written out with them
    r1, r2, r3 = (int(v) for v in ranks[:3])
    n1, n2, n3 = plan.n
    assert st["elements_compressed"] == n1 * r1 + r1 * n2 * r2 + r2 * n3 * r3 + plan.n_dir * r3
    # each TT step of the library truncates at budget gamma ||T|| / sqrt(7);
    # a direct TT-SVD at that per-step budget (gamma' = gamma sqrt(3/7)) can
    # keep no fewer ranks than an optimal one, so it bounds the library's
    direct = D.tt_svd(pl.stack4d(ops), tol * np.sqrt(3.0 / 7.0))
    assert all(0 < r <= d for r, d in zip(ranks[:3], direct.ranks)), (ranks, direct.ranks)


def test_tridiagonal_eigensolver_on_large_gram(native):
    """H-Tucker on a grid whose transfer-node Gram matrices exceed the size
    at which the library switches from Jacobi to Householder + QL: ranks and
    error still match the oracle."""
    K, L, tol = (8, 8, 8), 5, 1e-5
    plan = pl.Plan(K=K, L=L)
    ops = pl.operators(plan)
    comp = pl.compress(ops, "4d", "htucker", tol)
    r1, r2, r3, r4 = comp.parts.ranks[:4]
    assert min(r1 * r2, r3 * r4) > 96 or plan.n_dir > 96
    ranks, R = _host(native, K, L, "4d", "htucker", tol)
    assert tuple(int(v) for v in ranks) == tuple(comp.parts.ranks)
    T4 = np.stack(ops)
    assert abs(_rel(R, T4) - _rel(np.stack([comp.restore(p) for p in range(plan.n_dir)]), T4)) <= 1e-8


@pytest.mark.parametrize("fmt,dec,K,L,tol", [
    ("3d", "tucker", (6, 5, 7), 3, 1e-4),
    ("3d", "tt", (6, 5, 7), 3, 1e-3),
    ("4d", "tucker", (6, 5, 7), 3, 1e-4),
    ("4d", "htucker", (8, 8, 8), 4, 1e-3),
    ("4d", "tt", (6, 5, 7), 3, 1e-4),
])
def test_restore_error_statistic(native, fmt, dec, K, L, tol):
    """With FMMFFT_KEY_RESTORE_ERROR = 1 the set-up reports the FP64 relative
    error of its stored operator, sqrt(sum_p ||T_p - R_p||^2 / sum_p ||T_p||^2):
    it equals the error of the restored tensors against the oracle's
    operators and stays within the tolerance the decompositions guarantee."""
    plan = pl.Plan(K=K, L=L)
    T4 = np.stack(pl.operators(plan))
    h = native.fmmfft_plan_create(*K, 0.5, TWO_PI, L, FMT[fmt], DEC[dec], tol)
    try:
        assert native.fmmfft_plan_stats(h)["restore_rel_err"] == -1.0
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_RESTORE_ERROR, 1)
        _, R = native.fmmfft_compress_host(h)
        got = native.fmmfft_plan_stats(h)["restore_rel_err"]
        want = _rel(R, T4)
        assert 0.0 < got <= tol
        assert abs(got - want) <= 1e-9 + 1e-6 * want, (got, want)
    finally:
        native.fmmfft_plan_destroy(h)


def test_restore_error_is_opt_in(native):
    h = native.fmmfft_plan_create(6, 5, 7, 0.5, TWO_PI, 3, 3, 1, 1e-4)
    try:
        native.fmmfft_compress_host(h, restored=False)
        assert native.fmmfft_plan_stats(h)["restore_rel_err"] == -1.0
        for bad in (2, -1, 0.5):
            with pytest.raises(native.FmmfftError):
                native.fmmfft_plan_set(h, native.FMMFFT_KEY_RESTORE_ERROR, bad)
    finally:
        native.fmmfft_plan_destroy(h)
