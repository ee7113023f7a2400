"""GPU parity of the translation (Eq. 5) through the C ABI against the oracle.

Tolerances (relative L2 over the compared outputs):
  * complex128 path: 1e-10.  The library's FP64 operator generator and the
    oracle's agree to ~3e-12 (different Hankel-function recurrences); FP64
    FFT rounding adds ~1e-15 * log2(n).
  * complex64 path with an imported operator (same operator on both sides):
    2e-6.  FP32 rounding of the fields and operator (2^-24 ~ 6e-8 each) grows
    with the ~3 log2(n) butterfly levels of the forward and inverse 3D FFTs
    and the restore contractions; measured errors sit near 2e-7.
  * compressed operator produced by the library itself, against the oracle's
    uncompressed translation: tol + 1e-5, the acceptance bound (the truncation
    error of Alg. 1 is at most tol relative to the operator).
"""
import numpy as np
import pytest

from oracle import decomp as D
from oracle import pipeline as pl
from oracle import translate as tr
from seeded_inputs import field_spectra, field_spectra_rows

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def _gpu_translate(F, torch, h, S, nrhs, c128=False):
    dt = torch.complex128 if c128 else torch.complex64
    x = torch.from_numpy(np.ascontiguousarray(S.astype(np.complex128 if c128 else np.complex64))).to("cuda")
    y = torch.empty_like(x)
    F.fmmfft_translate(h, x, y, nrhs, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert F.fmmfft_poll_status(h) == 0
    return y.cpu().numpy().astype(np.complex128)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(F, K, L, fmt=0, decomp=0, tol=0.0, prec=None):
    h = F.fmmfft_plan_create(K[0], K[1], K[2], 0.5, TWO_PI, L, fmt, decomp, tol)
    if prec is not None:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
    return h


def _import_plain(F, h, ops):
    F.fmmfft_import_plain(h, np.stack(ops))


def _import_tucker(F, h, comp):
    ranks = np.array([t.ranks for t in comp.parts], dtype=np.int32)
    core = np.concatenate([t.core.ravel() for t in comp.parts])
    U = [np.concatenate([t.factors[i].ravel() for t in comp.parts]) for i in range(3)]
    F.fmmfft_import_tucker3d(h, ranks, core, *U)


def test_plain_c128_8cube_L5_all_fields(native, cuda):
    """Uncompressed complex128 translation, 8^3 boxes, L = 5, 72 directions, 1 RHS."""
    F, torch = native, cuda
    K, L, nrhs = (8, 8, 8), 5, 1
    h = _plan(F, K, L, prec=F.FMMFFT_PREC_C128)
    try:
        F.fmmfft_compress(h)
        plan = pl.Plan(K=K, L=L)
        assert F.fmmfft_plan_stats(h)["n_dir"] == plan.n_dir == 72
        S = field_spectra(1001, plan.n_dir, nrhs, K)
        out = _gpu_translate(F, torch, h, S, nrhs, c128=True)
        ops = pl.operators(plan)
        ref = pl.translate_with(lambda p: ops[p], S)
        assert _rel(out, ref) <= 1e-10
    finally:
        F.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("K,L,nrhs", [((5, 3, 6), 3, 2), ((3, 9, 2), 2, 1), ((16, 7, 9), 3, 1),
                                      ((4, 4, 4), 1, 3)])
def test_plain_c64_imported_operator(native, cuda, K, L, nrhs):
    """Same operator on both sides: isolates the kernels' FP32 arithmetic.
    Ragged box counts (not powers of two), anisotropic grids, several RHS."""
    F, torch = native, cuda
    plan = pl.Plan(K=K, L=L)
    ops = pl.operators(plan)
    h = _plan(F, K, L)
    try:
        _import_plain(F, h, ops)
        S = field_spectra(17 + sum(K), plan.n_dir, nrhs, K)
        out = _gpu_translate(F, torch, h, S, nrhs)
        ref = pl.translate_with(lambda p: ops[p], S)
        assert _rel(out, ref) <= 2e-6
        # and the brute-force Toeplitz sum for one field (Eq. 5 by definition)
        from oracle import operator as op
        kh = plan.directions()
        p = plan.n_dir // 2
        Tg = op.operator_grid(kh[p], K, plan.a, plan.k0, plan.L)
        Bd = tr.translate_field_direct(Tg, S[p, 1, nrhs - 1])
        assert _rel(out[p, 1, nrhs - 1], Bd) <= 2e-6
    finally:
        F.fmmfft_plan_destroy(h)


def test_all_near_offsets_give_zero(native, cuda):
    """K = 2 per axis: every offset is in the near shell, the far operator is
    identically zero and so must be every translated field."""
    F, torch = native, cuda
    h = _plan(F, (2, 2, 2), 2)
    try:
        F.fmmfft_compress(h)
        S = field_spectra(5, F.fmmfft_plan_stats(h)["n_dir"], 2, (2, 2, 2))
        out = _gpu_translate(F, torch, h, S, 2)
        assert np.count_nonzero(out) == 0
    finally:
        F.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("K,L,tol,nrhs", [((6, 5, 7), 4, 1e-3, 3), ((12, 12, 12), 5, 1e-5, 1)])
def test_tucker3d_imported_cores(native, cuda, K, L, tol, nrhs):
    """Oracle HOSVD cores restored on the GPU (Fig. 3(a)) vs the oracle's own
    restoration of the same cores: kernel arithmetic only."""
    F, torch = native, cuda
    plan = pl.Plan(K=K, L=L)
    ops = pl.operators(plan)
    comp = pl.compress(ops, "3d", "tucker", tol)
    h = _plan(F, K, L, 3, 1, tol)
    try:
        _import_tucker(F, h, comp)
        S = field_spectra(23, plan.n_dir, nrhs, K)
        out = _gpu_translate(F, torch, h, S, nrhs)
        ref = pl.translate_with(comp.restore, S)
        assert _rel(out, ref) <= 2e-6
    finally:
        F.fmmfft_plan_destroy(h)


def test_tucker3d_library_compression_acceptance(native, cuda):
    """The library's own compression (tol 1e-4) against the oracle's
    uncompressed FP64 translation: within tol + 1e-5."""
    F, torch = native, cuda
    K, L, tol, nrhs = (16, 16, 16), 6, 1e-4, 2
    h = _plan(F, K, L, 3, 1, tol)
    try:
        F.fmmfft_compress(h)
        st = F.fmmfft_plan_stats(h)
        assert 0.0 < st["saving"] < 1.0
        plan = pl.Plan(K=K, L=L)
        S = field_spectra(1002, plan.n_dir, nrhs, K)
        out = _gpu_translate(F, torch, h, S, nrhs)
        dirs = list(range(0, plan.n_dir, 7))
        ops = pl.operators(plan, dirs)
        ref = pl.translate_with(lambda p: ops[dirs.index(p)], S, dirs)
        assert _rel(out[dirs], ref[dirs]) <= tol + 1e-5
    finally:
        F.fmmfft_plan_destroy(h)


def _sampled_fields(F, torch, h, K, L, nrhs, seed, fields, restore=None):
    plan = pl.Plan(K=K, L=L)
    n_dir = plan.n_dir
    S = field_spectra(seed, n_dir, nrhs, K).astype(np.complex64)
    out = _gpu_translate(F, torch, h, S, nrhs)
    A = field_spectra_rows(seed, n_dir, nrhs, K, np.array(fields))
    errs = []
    for i, f in enumerate(fields):
        p, rem = divmod(f, 2 * nrhs)
        pol, r = divmod(rem, nrhs)
        T = pl.operators(plan, [p])[0] if restore is None else restore(p)
        ref = tr.translate_field_fft(T, A[i].astype(np.complex64).astype(np.complex128))
        errs.append(_rel(out[p, pol, r], ref))
    return errs


def test_benchmark_workload_tucker3d_32cube_L8(native, cuda):
    """The benchmark's workload and launch configuration: 32^3 boxes, L = 8,
    162 directions, 2 x 4 fields each, Tucker-3D at tol 1e-4.  Sampled fields
    (first, last and a middle one) against the oracle's FP64 translation."""
    F, torch = native, cuda
    K, L, tol, nrhs = (32, 32, 32), 8, 1e-4, 4
    h = _plan(F, K, L, 3, 1, tol)
    try:
        F.fmmfft_compress(h)
        n_fields = 162 * 2 * nrhs
        errs = _sampled_fields(F, torch, h, K, L, nrhs, 1002, [0, n_fields // 2 + 3, n_fields - 1])
        assert max(errs) <= tol + 1e-5, errs
    finally:
        F.fmmfft_plan_destroy(h)


def test_benchmark_workload_plain_32cube_L8(native, cuda):
    F, torch = native, cuda
    K, L, nrhs = (32, 32, 32), 8, 4
    h = _plan(F, K, L)
    try:
        F.fmmfft_compress(h)
        n_fields = 162 * 2 * nrhs
        errs = _sampled_fields(F, torch, h, K, L, nrhs, 1002, [5, n_fields - 6])
        assert max(errs) <= 1e-5, errs
    finally:
        F.fmmfft_plan_destroy(h)


def test_host_entry_point_matches_device_and_repeats(native, cuda):
    F, torch = native, cuda
    K, L, nrhs = (6, 6, 6), 3, 2
    h = _plan(F, K, L, 3, 1, 1e-4)
    try:
        F.fmmfft_compress(h)
        n_dir = F.fmmfft_plan_stats(h)["n_dir"]
        S = field_spectra(3, n_dir, nrhs, K).astype(np.complex64)
        a = _gpu_translate(F, torch, h, S, nrhs)
        b = _gpu_translate(F, torch, h, S, nrhs)
        assert np.array_equal(a, b)
        hin = torch.from_numpy(S).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        F.fmmfft_translate_host(h, hin, hout, nrhs, torch.cuda.current_stream())
        assert np.array_equal(hout.numpy().astype(np.complex128), a)
    finally:
        F.fmmfft_plan_destroy(h)


def test_invalid_calls_return_errors(native, cuda):
    F, torch = native, cuda
    K = (4, 4, 4)
    h = _plan(F, K, 2)
    try:
        F.fmmfft_compress(h)
        n_dir = F.fmmfft_plan_stats(h)["n_dir"]
        x = torch.zeros(n_dir * 2 * 64 * 2, dtype=torch.complex64, device="cuda")
        half = n_dir * 2 * 64
        for args in ((x, x, 1), (x[:half], x[1:half + 1], 1), (x[:half], x[half:], 0)):
            with pytest.raises(F.FmmfftError) as e:
                F.fmmfft_translate(h, *args)
            assert e.value.status == F.FMMFFT_ERR_INVALID_ARG
        F.fmmfft_translate(h, x[:half], x[half:], 1)
        torch.cuda.synchronize()
        assert F.fmmfft_poll_status(h) == 0
    finally:
        F.fmmfft_plan_destroy(h)


def test_unsupported_size_is_reported(native, cuda):
    """A z extent of 256 (Kz = 128) is outside the compiled y/z kernels."""
    F = native
    h = _plan(F, (4, 4, 128), 2)
    try:
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_compress(h)
        assert e.value.status == F.FMMFFT_ERR_UNSUPPORTED
    finally:
        F.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("K,L,nrhs", [((9, 17, 30), 2, 1), ((9, 12, 30), 2, 3)])
def test_ragged_planes_match_oracle(native, cuda, K, L, nrhs):
    """Ragged box counts whose FFT planes are 64 x 64 and 32 x 64, several RHS.
    Plain operator and Tucker-3D cores, both imported from the oracle."""
    F, torch = native, cuda
    plan = pl.Plan(K=K, L=L)
    ops = pl.operators(plan)
    comp = pl.compress(ops, "3d", "tucker", 1e-4)
    S = field_spectra(31 + nrhs, plan.n_dir, nrhs, K)
    hp = _plan(F, K, L)
    ht = _plan(F, K, L, 3, 1, 1e-4)
    try:
        _import_plain(F, hp, ops)
        _import_tucker(F, ht, comp)
        out_p = _gpu_translate(F, torch, hp, S, nrhs)
        out_t = _gpu_translate(F, torch, ht, S, nrhs)
        assert _rel(out_p, pl.translate_with(lambda p: ops[p], S)) <= 2e-6
        assert _rel(out_t, pl.translate_with(comp.restore, S)) <= 2e-6
    finally:
        F.fmmfft_plan_destroy(hp)
        F.fmmfft_plan_destroy(ht)


@pytest.mark.parametrize("K,L,fmt,dec,prec,blocks", [
    ((6, 6, 6), 3, 3, 1, 1, 5),        # Tucker-3D, 32 directions in blocks of 7 (last 4)
    ((6, 5, 7), 2, 4, 3, 2, 3),        # H-Tucker: pre-pass in the first block only, 3xTF32
    ((5, 64, 64), 1, 3, 1, 1, 3),      # 128 x 128 planes: persistent large-plane kernel
    ((4, 4, 4), 2, 0, 0, 0, 64),       # plain complex128, one direction per block
    ((6, 6, 6), 3, 4, 2, 1, 1),        # TT-4D, no pipelining
])
def test_host_pipeline_matches_device(native, cuda, K, L, fmt, dec, prec, blocks):
    """fmmfft_translate_host in direction blocks (copy-in, translate, copy-out
    overlapped) gives the device entry point's result bit for bit."""
    F, torch = native, cuda
    h = _plan(F, K, L, fmt, dec, 1e-4 if fmt else 0.0)
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
        F.fmmfft_compress(h)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_HOST_BLOCKS, blocks)
        n_dir = F.fmmfft_plan_stats(h)["n_dir"]
        nrhs = 2
        dt = np.complex128 if prec == 0 else np.complex64
        S = field_spectra(11, n_dir, nrhs, K).astype(dt)
        x = torch.from_numpy(S).cuda()
        y = torch.empty_like(x)
        F.fmmfft_translate(h, x, y, nrhs, torch.cuda.current_stream())
        torch.cuda.synchronize()
        ref = y.cpu().numpy()
        hin = torch.from_numpy(S).pin_memory()
        hout = torch.zeros_like(hin).pin_memory()
        for _ in range(2):
            F.fmmfft_translate_host(h, hin, hout, nrhs, torch.cuda.current_stream())
            assert np.array_equal(hout.numpy(), ref)
        assert F.fmmfft_poll_status(h) == 0
    finally:
        F.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("fmt,dec,prec", [(3, 1, 2), (0, 0, 1), (3, 2, 1), (4, 3, 1)])
def test_direction_shards_translate_their_block(native, cuda, fmt, dec, prec):
    """Shard plans (FMMFFT_KEY_DIR_FIRST / _COUNT) over three blocks of the
    directions: each translates its block of the fields; 3D formats and the
    plain operator match the whole plan bit for bit, the 4D format (which
    decomposes each block's own tensor) the oracle within tol + 1e-5."""
    from paper_2010_00520_gb300.replicas import direction_block
    F, torch = native, cuda
    K, L, nrhs, tol = (7, 6, 9), 3, 2, 1e-4
    h = _plan(F, K, L, fmt, dec, tol if fmt else 0.0, prec)
    try:
        F.fmmfft_compress(h)
        n_dir = F.fmmfft_plan_stats(h)["n_dir"]
        S = field_spectra(23, n_dir, nrhs, K).astype(np.complex64)
        whole = _gpu_translate(F, torch, h, S, nrhs)
    finally:
        F.fmmfft_plan_destroy(h)
    parts = []
    for r in range(3):
        first, count = direction_block(n_dir, 3, r)
        hs = _plan(F, K, L, fmt, dec, tol if fmt else 0.0, prec)
        try:
            F.fmmfft_plan_set(hs, F.FMMFFT_KEY_DIR_FIRST, first)
            F.fmmfft_plan_set(hs, F.FMMFFT_KEY_DIR_COUNT, count)
            F.fmmfft_compress(hs)
            assert F.fmmfft_plan_stats(hs)["n_dir"] == count
            parts.append(_gpu_translate(F, torch, hs, S[first:first + count], nrhs))
        finally:
            F.fmmfft_plan_destroy(hs)
    sharded = np.concatenate(parts)
    if fmt != 4:
        assert np.array_equal(sharded, whole)
    else:
        plan = pl.Plan(K=K, L=L)
        ops = pl.operators(plan)
        ref = pl.translate_with(lambda p: ops[p], S.astype(np.complex128))
        assert np.linalg.norm(sharded - ref) / np.linalg.norm(ref) <= tol + 1e-5


@pytest.mark.parametrize("fmt,dec,prec,bound", [(0, 0, 1, 2e-6), (3, 1, 2, 1e-4 + 1e-5)])
def test_maximum_extents_degenerate_L0(native, cuda, fmt, dec, prec, bound):
    """The largest grid the kernels take, 128 x 128 x 64 boxes (n = 256 x 256 x
    128, persistent large-plane kernel), at the degenerate L = 0: the operator
    is the isotropic monopole term for both directions of the grid.  Sampled
    fields against the oracle's FP64 translation."""
    F, torch = native, cuda
    K, L, nrhs = (128, 128, 64), 0, 1
    h = _plan(F, K, L, fmt, dec, 1e-4 if fmt else 0.0, prec)
    try:
        F.fmmfft_compress(h)
        st = F.fmmfft_plan_stats(h)
        assert st["n_dir"] == 2 and list(st["n"]) == [256, 256, 128] and st["large_planes"] == 1
        errs = _sampled_fields(F, torch, h, K, L, nrhs, 31, [0] if fmt == 0 else [3])
        assert max(errs) <= bound, errs
    finally:
        F.fmmfft_plan_destroy(h)


def test_smallest_grid(native, cuda):
    """K = 2 per axis (n = 4), every offset near except the far corners under the
    Chebyshev shell: only |d_i| <= 1, so the whole operator is zero; with the
    kappa = 0 rule (only d = 0 near) the far interactions are all there."""
    F, torch = native, cuda
    K, L, nrhs = (2, 2, 2), 1, 2
    for near, kappa in ((0, 4.0), (1, 0.0)):
        h = _plan(F, K, L, 0, 0, 0.0, 0)
        try:
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_NEAR_RULE, near)
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_KAPPA, kappa)
            F.fmmfft_compress(h)
            plan = pl.Plan(K=K, L=L, near_rule="chebyshev" if near == 0 else "kappa", kappa=kappa)
            S = field_spectra(5, plan.n_dir, nrhs, K)
            out = _gpu_translate(F, torch, h, S, nrhs, c128=True)
            ops = pl.operators(plan)
            ref = pl.translate_with(lambda p: ops[p], S)
            if near == 0:
                assert np.abs(out).max() == 0.0 and np.abs(ref).max() == 0.0
            else:
                assert _rel(out, ref) <= 1e-10
        finally:
            F.fmmfft_plan_destroy(h)
