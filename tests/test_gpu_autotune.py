"""GPU checks of the autotuner: it picks a schedule among the candidates
(x-pass block shape, tensor-core or CUDA-core restores and pre-pass, pre-pass
overlap), the translation keeps its results (to the 3xTF32 kernel-precision
bound), the choice lands in the tune cache and a fresh plan of the same shape
takes it from there; a batch can be tuned too."""
import os

import numpy as np
import pytest

from seeded_inputs import field_spectra

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def _rel(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(F, K=(9, 30, 32), L=2):
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, 3, 1, 1e-4)
    F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, F.FMMFFT_PREC_C64_3XTF32)
    F.fmmfft_compress(h)
    return h


def test_autotune_keeps_results_and_caches(native, cuda, tmp_path, monkeypatch):
    F, torch = native, cuda
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("FMMFFT_TUNE_CACHE", str(cache))
    K, nrhs = (9, 30, 32), 2
    h = _plan(F, K)
    h2 = None
    try:
        nd = F.fmmfft_plan_stats(h)["n_dir"]
        x = torch.from_numpy(field_spectra(5, nd, nrhs, K).astype(np.complex64)).to("cuda")
        y0, y1 = torch.empty_like(x), torch.empty_like(x)
        F.fmmfft_translate(h, x, y0, nrhs)
        F.fmmfft_autotune(h, nrhs, 3000.0)
        sched = F.fmmfft_plan_stats(h)["schedule"]
        assert sched[0] in (1, 2, 4) and sched[1] in (-1, 0) and sched[3] in (0, 1)
        F.fmmfft_translate(h, x, y1, nrhs)
        torch.cuda.synchronize()
        assert F.fmmfft_poll_status(h) == 0
        assert _rel(y1, y0) <= 5e-6
        lines = cache.read_text().strip().splitlines()
        assert len(lines) == 1 and f"nrhs={nrhs}" in lines[0]
        h2 = _plan(F, K)
        F.fmmfft_autotune(h2, nrhs, 3000.0)
        assert F.fmmfft_plan_stats(h2)["schedule"] == sched
        assert len(cache.read_text().strip().splitlines()) == 1     # served from the cache
    finally:
        F.fmmfft_plan_destroy(h)
        if h2:
            F.fmmfft_plan_destroy(h2)


def test_batch_autotune_then_translate(native, cuda, monkeypatch):
    F, torch = native, cuda
    monkeypatch.delenv("FMMFFT_TUNE_CACHE", raising=False)
    shapes = [(9, 30, 32), (6, 5, 7)]
    plans = [_plan(F, K, L) for K, L in zip(shapes, (2, 3))]
    try:
        xs, ys, refs, nr = [], [], [], [1, 2]
        for h, K, r in zip(plans, shapes, nr):
            nd = F.fmmfft_plan_stats(h)["n_dir"]
            xs.append(torch.from_numpy(field_spectra(9, nd, r, K).astype(np.complex64)).to("cuda"))
            ys.append(torch.empty_like(xs[-1]))
        b = F.fmmfft_batch_create(plans)
        try:
            F.fmmfft_batch_autotune(b, nr, 2000.0)
            for h, x, r in zip(plans, xs, nr):
                ref = torch.empty_like(x)
                F.fmmfft_translate(h, x, ref, r)
                refs.append(ref)
            s = torch.cuda.Stream()
            for _ in range(3):
                F.fmmfft_batch_translate(b, xs, ys, nr, s)
            s.synchronize()
            torch.cuda.synchronize()
            for y, ref in zip(ys, refs):
                assert torch.equal(y, ref)
        finally:
            F.fmmfft_batch_destroy(b)
    finally:
        for h in plans:
            F.fmmfft_plan_destroy(h)


def test_poll_straight_after_autotune(native, cuda):
    """The timing stream is private to the autotuner: a poll right after it
    (no translation in between) must neither wait on a destroyed stream nor
    see a status bit left by a candidate."""
    F, torch = native, cuda
    K, nrhs = (9, 30, 32), 2
    h = _plan(F, K)
    try:
        nd = F.fmmfft_plan_stats(h)["n_dir"]
        x = torch.from_numpy(field_spectra(6, nd, nrhs, K).astype(np.complex64)).to("cuda")
        y = torch.empty_like(x)
        F.fmmfft_translate(h, x, y, nrhs, torch.cuda.current_stream())
        F.fmmfft_autotune(h, nrhs, 2000.0)
        assert F.fmmfft_poll_status(h) == 0
        assert F.fmmfft_poll_status(h) == 0
    finally:
        F.fmmfft_plan_destroy(h)
