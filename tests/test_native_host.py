"""Host-side checks of the native library (no GPU needed).

* the shared library loads and exports every function include/fmmfft.h declares;
* argument validation of the plan life cycle;
* the library's own FP64 set-up (directions, operator of Eq. 7 embedded and
  FFT'ed as in Sec. II.B, HOSVD of Alg. 1) against the oracle.
"""
import os
import re

import numpy as np
import pytest

from oracle import decomp as D
from oracle import directions as dr
from oracle import pipeline as pl

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fmmfft.h")


def test_library_exports_every_declared_symbol(native):
    names = set(re.findall(r"^\s*(?:int|const char\*)\s+(fmmfft_\w+)\s*\(", open(HEADER).read(), re.M))
    assert len(names) >= 12
    assert names == set(native.EXPORTED)
    for n in names:
        assert hasattr(native.lib(), n), n


def test_status_strings(native):
    for s in (0, -1, -2, -3, -4, -5, -6, -7):
        assert native.fmmfft_status_string(s)
    assert native.fmmfft_status_string(-99) == "unknown status"


@pytest.mark.parametrize("args", [
    (1, 4, 4, 0.5, 6.28, 3, 0, 0, 0.0),        # K < 2
    (4, 4, 200, 0.5, 6.28, 3, 0, 0, 0.0),      # K > 128
    (4, 4, 4, -0.5, 6.28, 3, 0, 0, 0.0),       # a <= 0
    (4, 4, 4, 0.5, 0.0, 3, 0, 0, 0.0),         # k0 <= 0
    (4, 4, 4, 0.5, 6.28, -1, 0, 0, 0.0),       # L < 0
    (4, 4, 4, 0.5, 6.28, 3, 3, 0, 1e-3),       # 3D format without a decomposition
    (4, 4, 4, 0.5, 6.28, 3, 0, 1, 1e-3),       # decomposition without a format
    (4, 4, 4, 0.5, 6.28, 3, 3, 3, 1e-3),       # H-Tucker in the 3D format
    (4, 4, 4, 0.5, 6.28, 3, 3, 1, 0.0),        # tol 0 with a decomposition
    (4, 4, 4, 0.5, 6.28, 3, 7, 1, 1e-3),       # unknown format
])
def test_plan_create_rejects(native, args):
    with pytest.raises(native.FmmfftError) as e:
        native.fmmfft_plan_create(*args)
    assert e.value.status == native.FMMFFT_ERR_INVALID_ARG


def test_plan_set_and_translate_before_compress(native):
    h = native.fmmfft_plan_create(4, 4, 4, 0.5, 2 * np.pi, 3, 0, 0, 0.0)
    try:
        with pytest.raises(native.FmmfftError) as e:
            native.fmmfft_plan_set(h, 99, 1)
        assert e.value.status == native.FMMFFT_ERR_INVALID_ARG
        with pytest.raises(native.FmmfftError):
            native.fmmfft_plan_set(h, native.FMMFFT_KEY_PRECISION, 7)
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_NPHI_RULE, 1)
        assert native.fmmfft_plan_stats(h)["n_dir"] == 4 * 7
        with pytest.raises(native.FmmfftError) as e:
            native.fmmfft_translate(h, 16, 4096, 1, 0)
        assert e.value.status == native.FMMFFT_ERR_NOT_COMPRESSED
    finally:
        native.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("L,rule", [(3, 0), (5, 0), (8, 0), (6, 1)])
def test_directions_match_oracle(native, L, rule):
    h = native.fmmfft_plan_create(4, 4, 4, 0.5, 2 * np.pi, L, 0, 0, 0.0)
    try:
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_NPHI_RULE, rule)
        kh, w = native.fmmfft_plan_directions(h)
        kh2, w2 = dr.direction_grid(L, "benchmark" if rule == 0 else "paper")
        np.testing.assert_allclose(kh, kh2, atol=1e-14)
        np.testing.assert_allclose(w, w2, atol=1e-14)
        assert abs(w.sum() - 4 * np.pi) < 1e-12
    finally:
        native.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("K,L,near", [((4, 3, 5), 3, 0), ((8, 8, 8), 5, 0), ((6, 5, 4), 4, 1)])
def test_operator_generator_matches_oracle(native, K, L, near):
    h = native.fmmfft_plan_create(*K, 0.5, 2 * np.pi, L, 0, 0, 0.0)
    try:
        if near:
            native.fmmfft_plan_set(h, native.FMMFFT_KEY_NEAR_RULE, 1)
        plan = pl.Plan(K=K, L=L, near_rule="kappa" if near else "chebyshev")
        dirs = [0, plan.n_dir // 2, plan.n_dir - 1]
        ref = pl.operators(plan, dirs)
        for i, p in enumerate(dirs):
            T = native.fmmfft_operator_host(h, p)
            assert T.shape == plan.n
            assert np.linalg.norm(T - ref[i]) <= 1e-11 * np.linalg.norm(ref[i])
    finally:
        native.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("tol", [1e-3, 1e-4, 1e-6])
def test_hosvd_setup_matches_oracle(native, tol):
    K, L = (8, 8, 8), 5
    h = native.fmmfft_plan_create(*K, 0.5, 2 * np.pi, L, 3, 1, tol)
    try:
        plan = pl.Plan(K=K, L=L)
        for p in (1, 40):
            ranks, R = native.fmmfft_compress_direction_host(h, p)
            T = pl.operators(plan, [p])[0]
            tk = D.tucker_hosvd(T, tol)
            assert ranks == tk.ranks
            err = np.linalg.norm(R - T) / np.linalg.norm(T)
            assert err <= tol
            ref = np.linalg.norm(D.tucker_restore(tk) - T) / np.linalg.norm(T)
            assert abs(err - ref) <= 1e-9 + 1e-6 * ref
    finally:
        native.fmmfft_plan_destroy(h)


def test_plan_load_rejects_missing_and_foreign_files(native, tmp_path):
    with pytest.raises(native.FmmfftError) as e:
        native.fmmfft_plan_load(str(tmp_path / "missing.plan"))
    assert e.value.status == native.FMMFFT_ERR_IO
    bad = tmp_path / "bad.plan"
    bad.write_bytes(b"not a plan file at all, just some bytes")
    with pytest.raises(native.FmmfftError) as e:
        native.fmmfft_plan_load(str(bad))
    assert e.value.status == native.FMMFFT_ERR_INVALID_ARG
    h = native.fmmfft_plan_create(4, 4, 4, 0.5, 2 * np.pi, 2, 0, 0, 0.0)
    try:
        with pytest.raises(native.FmmfftError) as e:
            native.fmmfft_plan_save(h, str(tmp_path / "x.plan"))
        assert e.value.status == native.FMMFFT_ERR_NOT_COMPRESSED
    finally:
        native.fmmfft_plan_destroy(h)


def test_autotune_needs_a_compressed_plan(native):
    h = native.fmmfft_plan_create(4, 4, 4, 0.5, 2 * np.pi, 2, 0, 0, 0.0)
    try:
        with pytest.raises(native.FmmfftError) as e:
            native.fmmfft_autotune(h, 1, 100.0)
        assert e.value.status == native.FMMFFT_ERR_NOT_COMPRESSED
    finally:
        native.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("eps_r,pref,near", [(2 - 1j, 0, 0), (2 - 8j, 1, 1), (2.0, 1, 0)])
def test_operator_generator_matches_oracle_in_a_lossy_medium(native, eps_r, pref, near):
    """Sec. III.A.5: the library's FP64 operator with k = k0 sqrt(eps_r) (Hankel
    functions by upward recurrence in complex arithmetic) against the oracle's
    (terminating series)."""
    K, L = (6, 5, 7), 6
    h = native.fmmfft_plan_create(*K, 0.5, 2 * np.pi, L, 0, 0, 0.0)
    try:
        e = complex(eps_r)
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_EPS_R_RE, e.real)
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_EPS_R_IM, e.imag)
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_PREFACTOR, pref)
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_NEAR_RULE, near)
        plan = pl.Plan(K=K, L=L, eps_r=eps_r, prefactor="paper" if pref else "unit",
                       near_rule="kappa" if near else "chebyshev")
        dirs = [0, 17, plan.n_dir - 1]
        ref = pl.operators(plan, dirs)
        for i, p in enumerate(dirs):
            T = native.fmmfft_operator_host(h, p)
            assert np.linalg.norm(T - ref[i]) <= 1e-11 * np.linalg.norm(ref[i])
    finally:
        native.fmmfft_plan_destroy(h)


def test_medium_keys_validate(native):
    h = native.fmmfft_plan_create(4, 4, 4, 0.5, 2 * np.pi, 3, 0, 0, 0.0)
    try:
        for key, bad in ((native.FMMFFT_KEY_EPS_R_RE, 0.0), (native.FMMFFT_KEY_EPS_R_RE, -2.0),
                         (native.FMMFFT_KEY_EPS_R_IM, 0.5), (native.FMMFFT_KEY_EPS_R_RE, float("nan"))):
            with pytest.raises(native.FmmfftError) as e:
                native.fmmfft_plan_set(h, key, bad)
            assert e.value.status == native.FMMFFT_ERR_INVALID_ARG
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_EPS_R_IM, -8.0)
    finally:
        native.fmmfft_plan_destroy(h)


def _printed_counts():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "direction_counts.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            a, digits, er, ei, nd = line.split()[:5]
            rows.append((float(a), float(digits), complex(float(er), float(ei)), int(nd)))
    return rows


@pytest.mark.parametrize("row", _printed_counts())
def test_library_multipole_count_reproduces_printed_direction_counts(native, row):
    a, digits, eps_r, n_dir = row
    L = native.fmmfft_multipole_count(a, 2 * np.pi, digits, eps_r)
    assert (L + 1) * (2 * L + 1) == n_dir
    with pytest.raises(native.FmmfftError):
        native.fmmfft_multipole_count(a, 2 * np.pi, digits, complex(eps_r.real, 1.0))


def test_compress_host_records_statistics(native):
    """fmmfft_compress_host on a plan not yet compressed reports its ranks and
    memory saving (Sec. III: 1 - compressed / original) through plan_stats."""
    K, L = (8, 8, 8), 5
    h = native.fmmfft_plan_create(*K, 0.5, 2 * np.pi, L, 3, 1, 1e-4)
    try:
        r, _ = native.fmmfft_compress_host(h, restored=False)
        st = native.fmmfft_plan_stats(h)
        n = st["n"]
        stored = sum(int(a) * int(b) * int(c) + n[0] * int(a) + n[1] * int(b) + n[2] * int(c) for a, b, c in r)
        assert st["elements_compressed"] == stored
        assert st["elements_plain"] == n[0] * n[1] * n[2] * st["n_dir"]
        assert abs(st["saving"] - (1 - stored / st["elements_plain"])) < 1e-15
        assert list(st["max_rank"][:3]) == list(r.max(axis=0))
    finally:
        native.fmmfft_plan_destroy(h)


def test_shard_plan_directions_are_a_block_of_the_grid(native):
    L = 4
    h = native.fmmfft_plan_create(4, 4, 4, 0.5, 2 * np.pi, L, 0, 0, 0.0)
    try:
        kh, w = native.fmmfft_plan_directions(h)
        n = len(w)
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_DIR_FIRST, 7)
        assert native.fmmfft_plan_stats(h)["n_dir"] == n - 7           # count 0: to the end
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_DIR_COUNT, 11)
        kh2, w2 = native.fmmfft_plan_directions(h)
        assert native.fmmfft_plan_stats(h)["n_dir"] == 11
        assert np.array_equal(kh2, kh[7:18]) and np.array_equal(w2, w[7:18])
        for key, bad in ((native.FMMFFT_KEY_DIR_COUNT, n), (native.FMMFFT_KEY_DIR_FIRST, n),
                         (native.FMMFFT_KEY_DIR_FIRST, -1), (native.FMMFFT_KEY_DIR_COUNT, 2.5)):
            with pytest.raises(native.FmmfftError):
                native.fmmfft_plan_set(h, key, bad)
        assert native.fmmfft_plan_stats(h)["n_dir"] == 11                # unchanged by the rejects
        native.fmmfft_plan_set(h, native.FMMFFT_KEY_NPHI_RULE, 1)       # the block of the new grid
        kh3, _ = native.fmmfft_plan_directions(h)
        ref, _ = dr.direction_grid(L, "paper")
        assert np.allclose(kh3, ref[7:18], atol=1e-14)
    finally:
        native.fmmfft_plan_destroy(h)


def test_far_field_arguments_are_checked_before_any_launch(native):
    """fmmfft_aggregate / fmmfft_disaggregate reject bad arguments on the host,
    before touching a device (addresses below are never dereferenced)."""
    K, L = (4, 4, 4), 1
    h = native.fmmfft_plan_create(*K, 0.5, 2 * np.pi, L, 0, 0, 0.0)
    try:
        nd = native.fmmfft_plan_stats(h)["n_dir"]
        V, nb, nrhs = 64, 2, 1
        base = 1 << 40                                    # 256-byte aligned fake addresses
        P, I, A = base, base + (1 << 30), base + (2 << 30)
        cases = [
            (native.fmmfft_aggregate, (h, P, I, A, 0, nrhs), native.FMMFFT_ERR_INVALID_ARG),     # nb < 1
            (native.fmmfft_aggregate, (h, P, I, A, 49, nrhs), native.FMMFFT_ERR_UNSUPPORTED),    # nb > 48
            (native.fmmfft_aggregate, (h, P, I, A, nb, 0), native.FMMFFT_ERR_INVALID_ARG),       # nrhs < 1
            (native.fmmfft_aggregate, (h, P, I, A, nb, 5000), native.FMMFFT_ERR_INVALID_ARG),
            (native.fmmfft_aggregate, (h, 0, I, A, nb, nrhs), native.FMMFFT_ERR_INVALID_ARG),    # null
            (native.fmmfft_aggregate, (h, P + 4, I, A, nb, nrhs), native.FMMFFT_ERR_INVALID_ARG),  # misaligned
            # output overlapping the patterns / the coefficients
            (native.fmmfft_aggregate, (h, P, I, P + 8 * (nd * 2 * nb * V - 1), nb, nrhs),
             native.FMMFFT_ERR_INVALID_ARG),
            (native.fmmfft_aggregate, (h, P, I, I - 8, nb, nrhs), native.FMMFFT_ERR_INVALID_ARG),
            (native.fmmfft_disaggregate, (h, P, A, P, nb, nrhs), native.FMMFFT_ERR_INVALID_ARG),
            (native.fmmfft_disaggregate, (h, P, A, A + 8, nb, nrhs), native.FMMFFT_ERR_INVALID_ARG),
        ]
        for fn, args, status in cases:
            with pytest.raises(native.FmmfftError) as e:
                fn(*args)
            assert e.value.status == status, (fn.__name__, args[4:])
        with pytest.raises(native.FmmfftError) as e:
            native.fmmfft_aggregate(0, P, I, A, nb, nrhs)
        assert e.value.status == native.FMMFFT_ERR_INVALID_ARG
    finally:
        native.fmmfft_plan_destroy(h)


def test_host_blocks_key(native):
    h = native.fmmfft_plan_create(4, 4, 4, 0.5, 2 * np.pi, 1, 0, 0, 0.0)
    try:
        for ok in (0, 1, 12, 64):
            native.fmmfft_plan_set(h, native.FMMFFT_KEY_HOST_BLOCKS, ok)
        for bad in (-1, 65, 2.5):
            with pytest.raises(native.FmmfftError):
                native.fmmfft_plan_set(h, native.FMMFFT_KEY_HOST_BLOCKS, bad)
    finally:
        native.fmmfft_plan_destroy(h)
