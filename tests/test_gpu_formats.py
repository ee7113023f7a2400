"""GPU parity of the compressed formats beyond Tucker-3D: TT-3D (Fig. 4(a)),
Tucker-4D (Fig. 3(b)), H-Tucker (Fig. 3(c)) and TT-4D (Fig. 4(b)).

* imported oracle factors: the GPU restores the oracle's own decomposition;
  compared with the oracle translating with its restoration of the same
  factors (kernel arithmetic only): rel L2 <= 2e-6 in complex64, <= 1e-10 in
  complex128;
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
