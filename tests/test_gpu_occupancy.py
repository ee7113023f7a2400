"""GPU parity of the translation on partly occupied box grids (Sec. II.A:
empty boxes carry no sources and receive nothing), with the FFT lines of
empty x-rows pruned in both x passes.

Masks: the shell of boxes a meshed sphere occupies (interior empty, so whole
x-lines are empty) and random masks.  Against the oracle's masked translation
on the same inputs: complex128 1e-10, complex64 2e-6 (plain or FP32
restores), 5e-6 (3xTF32), compressed vs the uncompressed FP64 operator
tol + 1e-5.  Outputs at empty boxes are exactly zero; a full mask gives the
unmasked result bit for bit; clearing the mask restores the unmasked
translation; the host, allocation-free and fused-disaggregation entry points
honour the mask."""
import numpy as np
import pytest

from oracle import directions as dr
from oracle import farfield as ff
from oracle import pipeline as pl
from seeded_inputs import complex_gaussian, field_spectra, shell_occupancy

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _mask(K, kind, seed=3):
    if kind == "shell":
        return shell_occupancy(K)
    return np.random.default_rng(seed).random((K[2], K[1], K[0])) < 0.6


@pytest.mark.parametrize("K,L,nrhs,fmt,dec,prec,kind", [
    ((8, 8, 8), 3, 2, 0, 0, 0, "shell"),          # complex128 plain
    ((12, 10, 9), 3, 1, 0, 0, 1, "random"),       # ragged, complex64 plain
    ((16, 16, 16), 4, 2, 3, 1, 2, "shell"),       # Tucker-3D, 3xTF32
    ((9, 7, 11), 2, 3, 4, 3, 1, "shell"),         # H-Tucker, FP32 restores
    ((8, 64, 64), 1, 1, 3, 1, 2, "shell"),        # large-plane kernel (n2 x n3 = 128 x 128)
])
def test_masked_translation_matches_oracle(native, cuda, K, L, nrhs, fmt, dec, prec, kind):
    F, torch = native, cuda
    tol = 1e-4
    m = _mask(K, kind)
    assert 0 < m.sum() < m.size
    plan = pl.Plan(K=K, L=L)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, fmt, dec, tol if fmt else 0.0)
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
        F.fmmfft_compress(h)
        c128 = prec == 0
        cdt = np.complex128 if c128 else np.complex64
        S = field_spectra(21, plan.n_dir, nrhs, K).astype(cdt)
        x = torch.from_numpy(S).cuda()
        y_full, y_mask = torch.empty_like(x), torch.full_like(x, float("nan"))
        s = torch.cuda.current_stream()
        F.fmmfft_translate(h, x, y_full, nrhs, s)
        F.fmmfft_plan_set_occupancy(h, np.ones_like(m))
        y_ones = torch.empty_like(x)
        F.fmmfft_translate(h, x, y_ones, nrhs, s)
        F.fmmfft_plan_set_occupancy(h, m)
        F.fmmfft_translate(h, x, y_mask, nrhs, s)
        torch.cuda.synchronize()
        assert F.fmmfft_poll_status(h) == 0
        got = y_mask.cpu().numpy()
        assert np.array_equal(y_ones.cpu().numpy(), y_full.cpu().numpy())
        assert np.all(got[..., ~m] == 0)
        ops = pl.operators(plan)
        ref = pl.translate_occupied(lambda p: ops[p], S.astype(np.complex128), m)
        bound = 1e-10 if c128 else (tol + 1e-5 if fmt else 2e-6)
        assert _rel(got.astype(np.complex128), ref) <= bound
        # the unmasked translation of the input with its empty boxes zeroed
        xz = torch.from_numpy(np.where(m, S, 0).astype(cdt)).cuda()
        F.fmmfft_plan_set_occupancy(h, None)
        y_z = torch.empty_like(x)
        F.fmmfft_translate(h, xz, y_z, nrhs, s)
        y_again = torch.empty_like(x)
        F.fmmfft_translate(h, x, y_again, nrhs, s)
        torch.cuda.synchronize()
        gz = y_z.cpu().numpy()
        assert _rel(np.where(m, gz, 0).astype(np.complex128), got.astype(np.complex128)) <= (
            1e-12 if c128 else 1e-6)
        assert np.array_equal(y_again.cpu().numpy(), y_full.cpu().numpy())
    finally:
        F.fmmfft_plan_destroy(h)


def test_masked_host_noalloc_and_fused_disaggregation(native, cuda):
    F, torch = native, cuda
    K, L, nrhs, nb = (10, 8, 12), 2, 2, 5
    m = shell_occupancy(K)
    plan = pl.Plan(K=K, L=L)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, 0, 0, 0.0)
    try:
        F.fmmfft_compress(h)
        F.fmmfft_plan_set_occupancy(h, m)
        S = field_spectra(22, plan.n_dir, nrhs, K).astype(np.complex64)
        x = torch.from_numpy(S).cuda()
        y = torch.empty_like(x)
        s = torch.cuda.current_stream()
        F.fmmfft_translate(h, x, y, nrhs, s)
        y_na = torch.full_like(x, float("nan"))
        F.fmmfft_translate_noalloc(h, x, y_na, nrhs, s)
        hin = torch.from_numpy(S.copy()).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        F.fmmfft_translate_host(h, hin, hout, nrhs, s)
        box = (K[2], K[1], K[0])
        P = complex_gaussian(23, plan.n_dir * 2 * nb * int(np.prod(K))).reshape((plan.n_dir, 2, nb) + box)
        dP = torch.from_numpy(P.astype(np.complex64)).cuda()
        dy = torch.empty((nrhs, nb) + box, dtype=torch.complex64, device="cuda")
        F.fmmfft_translate_disaggregate(h, x, dP, dy, nb, nrhs, s)
        torch.cuda.synchronize()
        base = y.cpu().numpy()
        assert np.array_equal(y_na.cpu().numpy(), base)
        assert np.array_equal(hout.numpy(), base)
        ops = pl.operators(plan)
        B = pl.translate_occupied(lambda p: ops[p], S.astype(np.complex128), m)
        w = dr.direction_grid(L)[1]
        ref = ff.disaggregate(P.astype(np.complex64).astype(np.complex128), w, B)
        assert _rel(dy.cpu().numpy().astype(np.complex128), ref) <= 1e-5
        assert np.all(dy.cpu().numpy()[..., ~m] == 0)
        with pytest.raises(F.FmmfftError):
            F.fmmfft_plan_set_occupancy(h, np.ones(5, np.uint8))      # wrong size (binding check)
    finally:
        F.fmmfft_plan_destroy(h)
