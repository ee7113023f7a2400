"""GPU parity of the compressed formats beyond Tucker-3D: TT-3D (Fig. 4(a)),
Tucker-4D (Fig. 3(b)), H-Tucker (Fig. 3(c)) and TT-4D (Fig. 4(b)).

* imported oracle factors: the GPU restores the oracle's own decomposition;
  compared with the oracle translating with its restoration of the same
  factors (kernel arithmetic only): rel L2 <= 2e-6 in complex64 with FP32
  restores, <= 5e-6 with 3xTF32 tensor-core restores, <= 1e-10 in complex128.
  The 3xTF32 bound: each tensor-core product keeps big*big + small*big +
  big*small of the TF32 splits, a relative error near 2^-21 (~5e-7) per
  product; the H-Tucker restore chains four of them (E = C12 B, the core
  C_p = E V_p, H_p = U1 C_p, the slab) before the FP32 FFTs (~2e-7).  BF16x3
  (bf16 hi/lo splits) keeps about 16 bits per product (~1.5e-5 worst case,
  a few 1e-6 typical): bound 4e-5;
* the library's own compression against the oracle's uncompressed FP64
  translation: rel L2 <= tol + 1e-5 (acceptance bound).
"""
import numpy as np
import pytest

from oracle import pipeline as pl
from seeded_inputs import field_spectra

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi
FMT = {"3d": 3, "4d": 4}
DEC = {"tucker": 1, "tt": 2, "htucker": 3}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(F, torch, h, S, nrhs, c128=False):
    x = torch.from_numpy(np.ascontiguousarray(S.astype(np.complex128 if c128 else np.complex64))).to("cuda")
    y = torch.empty_like(x)
    F.fmmfft_translate(h, x, y, nrhs, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert F.fmmfft_poll_status(h) == 0
    return y.cpu().numpy().astype(np.complex128)


def _import(F, h, fmt, dec, P):
    c = lambda xs: np.concatenate([np.ravel(x) for x in xs])
    if fmt == "3d" and dec == "tt":
        F.fmmfft_import_tt3d(h, np.array([t.ranks for t in P], dtype=np.int32),
                             c([t.U1 for t in P]), c([t.cores[0] for t in P]), c([t.Ud for t in P]))
    elif dec == "tucker":
        F.fmmfft_import_tucker4d(h, np.array(P.ranks, dtype=np.int32), P.core, *P.factors)
    elif dec == "htucker":
        F.fmmfft_import_htucker(h, np.array(P.ranks, dtype=np.int32), *P.U, P.C12, P.C34, P.B)
    else:
        F.fmmfft_import_tt4d(h, np.array(P.ranks, dtype=np.int32), P.U1, P.cores[0], P.cores[1], P.Ud)


CASES = [("3d", "tt"), ("4d", "tucker"), ("4d", "htucker"), ("4d", "tt")]


@pytest.mark.parametrize("fmt,dec", CASES)
@pytest.mark.parametrize("K,L,nrhs,tol", [((6, 5, 7), 3, 2, 1e-4), ((9, 12, 30), 2, 1, 1e-3)])
def test_imported_factors_match_oracle(native, cuda, fmt, dec, K, L, nrhs, tol):
    F, torch = native, cuda
    plan = pl.Plan(K=K, L=L)
    ops = pl.operators(plan)
    comp = pl.compress(ops, fmt, dec, tol)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, FMT[fmt], DEC[dec], tol)
    try:
        _import(F, h, fmt, dec, comp.parts)
        S = field_spectra(51 + sum(K), plan.n_dir, nrhs, K)
        out = _run(F, torch, h, S, nrhs)
        assert _rel(out, pl.translate_with(comp.restore, S)) <= 2e-6
    finally:
        F.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("fmt,dec", [("4d", "htucker"), ("3d", "tt")])
def test_imported_factors_complex128(native, cuda, fmt, dec):
    F, torch = native, cuda
    K, L, nrhs, tol = (6, 5, 7), 3, 1, 1e-6
    plan = pl.Plan(K=K, L=L)
    ops = pl.operators(plan)
    comp = pl.compress(ops, fmt, dec, tol)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, FMT[fmt], DEC[dec], tol)
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, F.FMMFFT_PREC_C128)
        _import(F, h, fmt, dec, comp.parts)
        S = field_spectra(61, plan.n_dir, nrhs, K)
        out = _run(F, torch, h, S, nrhs, c128=True)
        assert _rel(out, pl.translate_with(comp.restore, S)) <= 1e-10
    finally:
        F.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("fmt,dec", CASES)
def test_library_compression_acceptance(native, cuda, fmt, dec):
    """The library's own compression at tol 1e-4 against the oracle's
    uncompressed FP64 translation."""
    F, torch = native, cuda
    K, L, nrhs, tol = (12, 10, 9), 4, 2, 1e-4
    plan = pl.Plan(K=K, L=L)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, FMT[fmt], DEC[dec], tol)
    try:
        F.fmmfft_compress(h)
        st = F.fmmfft_plan_stats(h)
        assert 0.0 < st["saving"] < 1.0
        S = field_spectra(71, plan.n_dir, nrhs, K)
        out = _run(F, torch, h, S, nrhs)
        ops = pl.operators(plan)
        ref = pl.translate_with(lambda p: ops[p], S)
        assert _rel(out, ref) <= tol + 1e-5
    finally:
        F.fmmfft_plan_destroy(h)


def _import_any(F, h, fmt, dec, comp):
    if fmt == "3d" and dec == "tucker":
        P = comp.parts
        F.fmmfft_import_tucker3d(h, np.array([t.ranks for t in P], dtype=np.int32),
                                 np.concatenate([t.core.ravel() for t in P]),
                                 *[np.concatenate([t.factors[i].ravel() for t in P]) for i in range(3)])
    else:
        _import(F, h, fmt, dec, comp.parts)


@pytest.mark.parametrize("prec,bound", [(2, 5e-6), (3, 4e-5), (4, 3e-3)])
@pytest.mark.parametrize("fmt,dec", [("3d", "tucker")] + CASES)
@pytest.mark.parametrize("K", [(9, 30, 32), (9, 12, 16), (7, 30, 11)])
def test_tensor_core_restore_matches_oracle(native, cuda, fmt, dec, prec, bound, K, record_property):
    """FMMFFT_PREC_C64_3XTF32 / BF16X3 / TF32 on y-z planes of 64 x 64, 32 x 32
    and 64 x 32 (one partly filled tensor-core tile): the slab restores run on
    the tensor cores (tcgen05).  Same imported factors as the oracle; the split
    products keep the bounds of the CUDA-core path; the single TF32 product
    (the ablation) rounds each operand to 11 bits, about 5e-4 per product,
    and chains two to four of them: bound 3e-3.  Measured maxima over these
    cases: 3xTF32 2.2e-6, BF16x3 1.1e-5, TF32 7.0e-4 (recorded per case as
    the rel_err property)."""
    F, torch = native, cuda
    L, nrhs, tol = 2, 2, 1e-4
    plan = pl.Plan(K=K, L=L)
    assert plan.n[1:] in ((64, 64), (32, 32), (64, 32))
    ops = pl.operators(plan)
    comp = pl.compress(ops, fmt, dec, tol)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, FMT[fmt], DEC[dec], tol)
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
        _import_any(F, h, fmt, dec, comp)
        assert F.fmmfft_plan_stats(h)["restore_on_tensor_cores"] == prec - 1
        S = field_spectra(81 + DEC[dec], plan.n_dir, nrhs, K)
        out = _run(F, torch, h, S, nrhs)
        err = _rel(out, pl.translate_with(comp.restore, S))
        record_property("rel_err", err)
        assert err <= bound
    finally:
        F.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("prec", [2, 3])
def test_tensor_core_restore_benchmark_workload(native, cuda, prec):
    """The benchmark's compressed arm (32^3 boxes, L = 8, Tucker-3D tol 1e-4,
    3xTF32 restores on the tensor cores, 2 x 4 fields per direction), sampled
    fields against the oracle's uncompressed FP64 translation."""
    F, torch = native, cuda
    K, L, tol, nrhs = (32, 32, 32), 8, 1e-4, 4
    plan = pl.Plan(K=K, L=L)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, 3, 1, tol)
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
        F.fmmfft_compress(h)
        assert F.fmmfft_plan_stats(h)["restore_on_tensor_cores"] == prec - 1
        S = field_spectra(1002, plan.n_dir, nrhs, K).astype(np.complex64)
        out = _run(F, torch, h, S, nrhs)
        from seeded_inputs import field_spectra_rows
        from oracle import translate as tr
        fields = [0, 7, 648 + 3, 1295]
        A = field_spectra_rows(1002, plan.n_dir, nrhs, K, np.array(fields))
        for i, f in enumerate(fields):
            p, rem = divmod(f, 2 * nrhs)
            pol, r = divmod(rem, nrhs)
            T = pl.operators(plan, [p])[0]
            ref = tr.translate_field_fft(T, A[i].astype(np.complex64).astype(np.complex128))
            assert _rel(out[p, pol, r], ref) <= tol + 1e-5
    finally:
        F.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("eps_r", [2 - 2j, 2 - 8j])
@pytest.mark.parametrize("fmt,dec,prec", [("none", None, 0), ("none", None, 1), ("3d", "tucker", 2),
                                          ("4d", "htucker", 1)])
def test_lossy_medium_translation(native, cuda, eps_r, fmt, dec, prec):
    """Sec. III.A.5 (Table IV): operators of a lossy medium, k = k0 sqrt(eps_r),
    through the same kernels; against the oracle's uncompressed FP64 translation
    (plain: <= 1e-10 in complex128, <= 2e-6 in complex64; compressed at tol
    1e-4: <= tol + 1e-5)."""
    F, torch = native, cuda
    K, L, nrhs, tol = (8, 6, 10), 4, 2, 1e-4
    plan = pl.Plan(K=K, L=L, eps_r=eps_r)
    if fmt == "none":
        h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, 0, 0, 0.0)
    else:
        h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, FMT[fmt], DEC[dec], tol)
    try:
        e = complex(eps_r)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_EPS_R_RE, e.real)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_EPS_R_IM, e.imag)
        F.fmmfft_compress(h)
        S = field_spectra(91, plan.n_dir, nrhs, K)
        out = _run(F, torch, h, S, nrhs, c128=(prec == 0))
        ops = pl.operators(plan)
        ref = pl.translate_with(lambda p: ops[p], S)
        bound = {"none": 1e-10 if prec == 0 else 2e-6}.get(fmt, tol + 1e-5)
        assert _rel(out, ref) <= bound
        if fmt != "none":
            assert F.fmmfft_plan_stats(h)["saving"] > 0.0
    finally:
        F.fmmfft_plan_destroy(h)
