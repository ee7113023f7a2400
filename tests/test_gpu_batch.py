"""GPU checks of the batch API: several independent plans with uneven grids,
multipole counts, formats and RHS counts translated by one call, forked over
internal streams; repeated calls with the same buffers are captured once as a
CUDA graph and replayed.  Every instance must equal its own fmmfft_translate
result exactly (same kernels, same inputs) on the eager call, the capturing
call and the replays, and one instance is checked against the oracle."""
import numpy as np
import pytest

from oracle import pipeline as pl
from seeded_inputs import field_spectra

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def test_batch_matches_single_translations_and_graph_replays(native, cuda):
    F, torch = native, cuda
    rng = np.random.default_rng(2024)
    specs = []
    for i in range(6):
        K = tuple(int(k) for k in rng.integers(5, 13, size=3))
        L = int(rng.integers(2, 5))
        fmt, dec, tol = [(3, 1, 1e-4), (0, 0, 0.0), (3, 2, 1e-4)][i % 3]
        specs.append((K, L, fmt, dec, tol, int(rng.integers(1, 4))))
    plans, xs, ys, refs, nrhs = [], [], [], [], []
    stream = torch.cuda.Stream()
    try:
        for (K, L, fmt, dec, tol, r) in specs:
            h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, fmt, dec, tol)
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, F.FMMFFT_PREC_C64_3XTF32 if fmt else F.FMMFFT_PREC_C64)
            F.fmmfft_compress(h)
            plans.append(h)
            nd = F.fmmfft_plan_stats(h)["n_dir"]
            xs.append(torch.from_numpy(field_spectra(300 + len(plans), nd, r, K).astype(np.complex64)).to("cuda"))
            ys.append(torch.empty_like(xs[-1]))
            nrhs.append(r)
        with torch.cuda.stream(stream):
            for h, x, r in zip(plans, xs, nrhs):
                ref = torch.empty_like(x)
                F.fmmfft_translate(h, x, ref, r, stream)
                refs.append(ref)
        stream.synchronize()
        b = F.fmmfft_batch_create(plans)
        try:
            for call in range(4):          # eager, capture, replay, replay
                for y in ys:
                    y.fill_(float("nan"))
                stream.synchronize()
                F.fmmfft_batch_translate(b, xs, ys, nrhs, stream)
                stream.synchronize()
                for h, y, ref in zip(plans, ys, refs):
                    assert F.fmmfft_poll_status(h) == 0
                    assert torch.equal(y, ref), call
            # new inputs in the same buffers: the replayed graph reads them
            xs[0].copy_(torch.flip(xs[0], dims=[0]))
            with torch.cuda.stream(stream):
                F.fmmfft_translate(plans[0], xs[0], refs[0], nrhs[0], stream)
            F.fmmfft_batch_translate(b, xs, ys, nrhs, stream)
            stream.synchronize()
            assert torch.equal(ys[0], refs[0])
        finally:
            F.fmmfft_batch_destroy(b)
        # instance 1 (plain operator) against the oracle
        K, L = specs[1][0], specs[1][1]
        plan = pl.Plan(K=K, L=L)
        ops = pl.operators(plan)
        S = xs[1].cpu().numpy().astype(np.complex128)
        ref = pl.translate_with(lambda p: ops[p], S)
        out = ys[1].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 2e-6
    finally:
        for h in plans:
            F.fmmfft_plan_destroy(h)


def test_batch_rejects_bad_arguments(native, cuda):
    F, torch = native, cuda
    h = F.fmmfft_plan_create(4, 4, 4, 0.5, TWO_PI, 2, 0, 0, 0.0)
    try:
        F.fmmfft_compress(h)
        b = F.fmmfft_batch_create([h])
        try:
            x = torch.zeros(F.fmmfft_plan_stats(h)["n_dir"] * 2 * 64, dtype=torch.complex64, device="cuda")
            with pytest.raises(F.FmmfftError) as e:
                F.fmmfft_batch_translate(b, [x], [x], [1])      # aliasing
            assert e.value.status == F.FMMFFT_ERR_INVALID_ARG
            with pytest.raises(F.FmmfftError):
                F.fmmfft_batch_translate(b, [x], [torch.empty_like(x)], [0])
        finally:
            F.fmmfft_batch_destroy(b)
        with pytest.raises(F.FmmfftError):
            F.fmmfft_batch_create([])
    finally:
        F.fmmfft_plan_destroy(h)
