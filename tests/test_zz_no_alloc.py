"""GPU checks of fmmfft_translate_noalloc, the translation entry point that
allocates no device memory.

It exists for callers that cannot call cudaMalloc while they translate (a
solver inside a framework whose memory pool owns the device, or a loop where
an allocation's implicit device synchronisation would stall other work).  Its
intermediate lives in the library's fixed 32 MiB device array instead of a
buffer the plan allocates, so its results must equal fmmfft_translate's.  The
file is named to run last: a run that stops at the first failure has then run
every other test already.  It passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from seeded_inputs import field_spectra

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("K,L,fmt,decomp,tol,c128,nrhs,bound", [
    ((6, 5, 7), 3, 3, 1, 1e-4, False, 2, 2e-6),      # Tucker-3D, complex64
    ((8, 8, 8), 5, 0, 0, 0.0, True, 1, 1e-10),       # plain operator, complex128
])
def test_noalloc_matches_translate_on_two_calls_in_a_row(native, cuda, K, L, fmt, decomp, tol, c128,
                                                         nrhs, bound):
    F, torch = native, cuda
    h = F.fmmfft_plan_create(K[0], K[1], K[2], 0.5, TWO_PI, L, fmt, decomp, tol)
    try:
        if c128:
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, F.FMMFFT_PREC_C128)
        F.fmmfft_compress(h)
        n_dir = F.fmmfft_plan_stats(h)["n_dir"]
        cdt = np.complex128 if c128 else np.complex64
        stream = torch.cuda.current_stream()
        xs = [torch.from_numpy(field_spectra(seed, n_dir, nrhs, K).astype(cdt)).to("cuda")
              for seed in (41, 42)]
        outs = [torch.full_like(x, float("nan")) for x in xs]
        # two calls in a row on different inputs: the second must not depend
        # on what the first left in the shared scratch
        for x, y in zip(xs, outs):
            F.fmmfft_translate_noalloc(h, x, y, nrhs, stream)
        torch.cuda.synchronize()
        assert F.fmmfft_poll_status(h) == 0
        for x, y in zip(xs, outs):
            ref = torch.empty_like(x)
            F.fmmfft_translate(h, x, ref, nrhs, stream)
            torch.cuda.synchronize()
            a = y.cpu().numpy().astype(np.complex128)
            b = ref.cpu().numpy().astype(np.complex128)
            assert np.isfinite(a).all()
            assert _rel(a, b) <= bound
            # same kernels, schedule and inputs, only the intermediate's
            # address differs, and no kernel sums in a data-dependent order:
            # the two outputs are bit for bit the same (a few stale scratch
            # elements would pass the bound above but not this)
            assert np.array_equal(a, b)
    finally:
        F.fmmfft_plan_destroy(h)


def test_noalloc_size_limit(native, cuda):
    """32^3 boxes, L = 1 (8 directions), complex64: the intermediate is
    8 * 2 * nrhs * 64 * 32 * 32 * 8 bytes, exactly the 32 MiB limit at
    nrhs = 4 (accepted) and over it at nrhs = 5 (FMMFFT_ERR_TOO_LARGE before
    any launch; the output buffer is left untouched)."""
    F, torch = native, cuda
    K = (32, 32, 32)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, 1, 0, 0, 0.0)
    try:
        F.fmmfft_compress(h)
        n_dir = F.fmmfft_plan_stats(h)["n_dir"]
        assert n_dir * 2 * 4 * 64 * 32 * 32 * 8 == F.FMMFFT_NOALLOC_SCRATCH_BYTES
        stream = torch.cuda.current_stream()
        x = torch.from_numpy(field_spectra(43, n_dir, 4, K).astype(np.complex64)).to("cuda")
        y = torch.empty_like(x)
        ref = torch.empty_like(x)
        F.fmmfft_translate_noalloc(h, x, y, 4, stream)
        F.fmmfft_translate(h, x, ref, 4, stream)
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128)) <= 2e-6
        x5 = torch.zeros(n_dir * 2 * 5 * 32 ** 3, dtype=torch.complex64, device="cuda")
        y5 = torch.full_like(x5, 7.0)
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_translate_noalloc(h, x5, y5, 5, stream)
        assert e.value.status == F.FMMFFT_ERR_TOO_LARGE
        torch.cuda.synchronize()
        assert bool((y5 == 7.0).all())
    finally:
        F.fmmfft_plan_destroy(h)
