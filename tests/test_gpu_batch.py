"""GPU checks of the batch API: several independent plans with uneven grids,
multipole counts, formats and RHS counts translated by one call.  Complex64
instances run in launches shared by all instances of a shape class (one
launch per phase and class); complex128 ones run their own
launches on internal streams.  Repeated calls with the same buffers are
captured once as a CUDA graph and replayed.  Every instance must equal its
own fmmfft_translate result exactly (same device code, same inputs) on the
eager call, the capturing call and the replays, and instances are checked
against the oracle."""
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
    # one complex128 instance runs its own launches beside the shared ones
    specs.append(((6, 7, 5), 2, 0, 0, 0.0, 2))
    plans, xs, ys, refs, nrhs = [], [], [], [], []
    stream = torch.cuda.Stream()
    try:
        for j, (K, L, fmt, dec, tol, r) in enumerate(specs):
            c128 = j == len(specs) - 1
            h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, fmt, dec, tol)
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, F.FMMFFT_PREC_C128 if c128 else
                              F.FMMFFT_PREC_C64_3XTF32 if fmt else F.FMMFFT_PREC_C64)
            F.fmmfft_compress(h)
            plans.append(h)
            nd = F.fmmfft_plan_stats(h)["n_dir"]
            xs.append(torch.from_numpy(field_spectra(300 + len(plans), nd, r, K)
                                       .astype(np.complex128 if c128 else np.complex64)).to("cuda"))
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
                assert F.fmmfft_batch_shared_count(b) == len(plans) - 1
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


def test_shared_launch_batch_of_uneven_instances(native, cuda, monkeypatch):
    """20 instances of uneven grids (K_i drawn from 8..24 per axis, so FFT
    extents 16, 32 or 64), multipole counts L in 1..4, Tucker-3D at tol 1e-4
    with 3xTF32 or FP32 restores, H-Tucker and plain operators, 1..3 RHS: all
    of them run in the shared launches (one per phase and shape class), equal their own single translations bit for bit, equal the batch
    with one launch sequence per instance (FMMFFT_BATCH_SEPARATE=1) bit for
    bit, and sampled fields lie within tol + 1e-5 (plain: 2e-6) of the
    oracle's FP64 translation."""
    F, torch = native, cuda
    rng = np.random.default_rng(77)
    specs = []
    for i in range(20):
        K = tuple(int(k) for k in rng.integers(8, 25, size=3))
        L = int(rng.integers(1, 5))
        fmt, dec, tol, prec = [(3, 1, 1e-4, 2), (0, 0, 0.0, 1), (3, 1, 1e-4, 1), (4, 3, 1e-4, 2)][i % 4]
        specs.append((K, L, fmt, dec, tol, prec, int(rng.integers(1, 4))))
    plans, xs, refs, nrhs = [], [], [], []
    stream = torch.cuda.Stream()
    try:
        for (K, L, fmt, dec, tol, prec, r) in specs:
            h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, fmt, dec, tol)
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
            F.fmmfft_compress(h)
            plans.append(h)
            nd = F.fmmfft_plan_stats(h)["n_dir"]
            xs.append(torch.from_numpy(field_spectra(500 + len(plans), nd, r, K).astype(np.complex64)).to("cuda"))
            nrhs.append(r)
        with torch.cuda.stream(stream):
            for h, x, r in zip(plans, xs, nrhs):
                ref = torch.empty_like(x)
                F.fmmfft_translate(h, x, ref, r, stream)
                refs.append(ref)
        stream.synchronize()
        outs = {}
        for mode in ("shared", "separate"):
            monkeypatch.setenv("FMMFFT_BATCH_SEPARATE", "1" if mode == "separate" else "0")
            b = F.fmmfft_batch_create(plans)
            try:
                ys = [torch.full_like(x, float("nan")) for x in xs]
                for call in range(3):                    # eager, capture, replay
                    F.fmmfft_batch_translate(b, xs, ys, nrhs, stream)
                    stream.synchronize()
                    for h, y, ref in zip(plans, ys, refs):
                        assert F.fmmfft_poll_status(h) == 0
                        assert torch.equal(y, ref), (mode, call)
                shared = F.fmmfft_batch_shared_count(b)
                assert shared == (len(plans) if mode == "shared" else 0), shared
                outs[mode] = [y.clone() for y in ys]
            finally:
                F.fmmfft_batch_destroy(b)
        for a, c in zip(outs["shared"], outs["separate"]):
            assert torch.equal(a, c)
        # sampled instances against the oracle's uncompressed FP64 translation
        from oracle import translate as tr
        for i in (0, 1, 2, 3, 7):
            K, L, fmt, dec, tol, prec, r = specs[i]
            plan = pl.Plan(K=K, L=L)
            S = xs[i].cpu().numpy().astype(np.complex128)
            out = outs["shared"][i].cpu().numpy().astype(np.complex128)
            dirs = [0, plan.n_dir - 1]
            got, want = [], []
            for p in dirs:
                T = pl.operators(plan, [p])[0]
                for pol in range(2):
                    want.append(tr.translate_field_fft(T, S[p, pol, 0]))
                    got.append(out[p, pol, 0])
            err = np.linalg.norm(np.stack(got) - np.stack(want)) / np.linalg.norm(np.stack(want))
            assert err <= (tol + 1e-5 if fmt else 2e-6), (i, err)
    finally:
        for h in plans:
            F.fmmfft_plan_destroy(h)


def test_batch_class_larger_than_one_descriptor_table(native, cuda):
    """130 small instances of one shape class (grids 5..8 per axis, so FFT
    extents of 16, plain operator, L = 1): more instances than one x-pass
    launch carries in its parameters, so the class's x passes run as several
    launches.  Every instance equals its own translation bit for bit."""
    F, torch = native, cuda
    rng = np.random.default_rng(5)
    plans, xs, refs, nrhs = [], [], [], []
    stream = torch.cuda.Stream()
    try:
        for j in range(130):
            K = tuple(int(k) for k in rng.integers(5, 9, size=3))
            h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, 1, 0, 0, 0.0)
            F.fmmfft_compress(h)
            plans.append(h)
            r = 1 + j % 2
            nd = F.fmmfft_plan_stats(h)["n_dir"]
            xs.append(torch.from_numpy(field_spectra(900 + j, nd, r, K).astype(np.complex64)).to("cuda"))
            nrhs.append(r)
        with torch.cuda.stream(stream):
            for h, x, r in zip(plans, xs, nrhs):
                ref = torch.empty_like(x)
                F.fmmfft_translate(h, x, ref, r, stream)
                refs.append(ref)
        stream.synchronize()
        b = F.fmmfft_batch_create(plans)
        try:
            ys = [torch.full_like(x, float("nan")) for x in xs]
            for call in range(2):
                F.fmmfft_batch_translate(b, xs, ys, nrhs, stream)
                stream.synchronize()
                assert F.fmmfft_batch_shared_count(b) == len(plans)
                for h, y, ref in zip(plans, ys, refs):
                    assert F.fmmfft_poll_status(h) == 0
                    assert torch.equal(y, ref), call
        finally:
            F.fmmfft_batch_destroy(b)
    finally:
        for h in plans:
            F.fmmfft_plan_destroy(h)
