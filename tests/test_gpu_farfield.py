"""GPU parity of the far-field steps (Eqs. 4 and 6) against the oracle.

Random patterns, coefficients and spectra (seeded complex Gaussians), ragged
box counts (not multiples of the 128-box tiles), basis-function and RHS counts
off the kernels' tile sizes, odd direction counts.  Bounds: complex64 rel L2
2e-6 for aggregation (sums of nb FP32 products), 1e-5 for disaggregation (sums
of 2 n_dir products, sqrt(2 n_dir) eps growth); complex128 1e-12.  The chain
aggregate -> translate -> disaggregate is checked against the oracle's chain.
"""
import numpy as np
import pytest

from oracle import directions as dr
from oracle import farfield as ff
from oracle import pipeline as pl
from seeded_inputs import complex_gaussian

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cg(seed, shape):
    return complex_gaussian(seed, int(np.prod(shape))).reshape(shape)


def _dev(torch, x, c128):
    return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex128 if c128 else np.complex64))).cuda()


@pytest.mark.parametrize("c128", [False, True])
@pytest.mark.parametrize("K,L,nphi,nb,nrhs", [((5, 7, 3), 2, 1, 3, 5), ((8, 8, 8), 3, 0, 16, 4),
                                              ((9, 6, 4), 2, 0, 48, 1), ((4, 4, 4), 0, 1, 1, 2),
                                              ((16, 12, 10), 4, 1, 5, 3)])
def test_aggregate_and_disaggregate_match_oracle(native, cuda, c128, K, L, nphi, nb, nrhs):
    F, torch = native, cuda
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, 0, 0, 0.0)
    try:
        if c128:
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, F.FMMFFT_PREC_C128)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_NPHI_RULE, nphi)
        nd = F.fmmfft_plan_stats(h)["n_dir"]
        _, w = F.fmmfft_plan_directions(h)
        box = (K[2], K[1], K[0])
        P = _cg(41 + nb, (nd, 2, nb) + box)
        I = _cg(42 + nb, (nrhs, nb) + box)
        Bs = _cg(43 + nb, (nd, 2, nrhs) + box)
        dP, dI, dB = _dev(torch, P, c128), _dev(torch, I, c128), _dev(torch, Bs, c128)
        dA = torch.empty_like(dB)
        dy = torch.empty_like(dI)
        s = torch.cuda.current_stream()
        F.fmmfft_aggregate(h, dP, dI, dA, nb, nrhs, s)
        F.fmmfft_disaggregate(h, dP, dB, dy, nb, nrhs, s)
        torch.cuda.synchronize()
        A, y = dA.cpu().numpy(), dy.cpu().numpy()
        assert _rel(A, ff.aggregate(P, I)) <= (1e-12 if c128 else 2e-6)
        assert _rel(y, ff.disaggregate(P, w, Bs)) <= (1e-12 if c128 else 1e-5)
    finally:
        F.fmmfft_plan_destroy(h)


@pytest.mark.parametrize("fmt,dec,prec", [(0, 0, 0), (3, 1, 2)])
def test_far_field_matvec_chain_matches_oracle(native, cuda, fmt, dec, prec):
    """Eq. 4 -> Eq. 5 -> Eq. 6 on the device (plain complex128, and Tucker-3D
    with 3xTF32 restores) against the oracle's chain on the same inputs."""
    F, torch = native, cuda
    K, L, nb, nrhs, tol = (10, 8, 12), 3, 6, 2, 1e-4
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, fmt, dec, tol)
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
        F.fmmfft_compress(h)
        c128 = prec == 0
        nd = F.fmmfft_plan_stats(h)["n_dir"]
        _, w = F.fmmfft_plan_directions(h)
        box = (K[2], K[1], K[0])
        P = _cg(51, (nd, 2, nb) + box)
        I = _cg(52, (nrhs, nb) + box)
        dP, dI = _dev(torch, P, c128), _dev(torch, I, c128)
        dA = torch.empty((nd, 2, nrhs) + box, dtype=dP.dtype, device="cuda")
        dB = torch.empty_like(dA)
        dy = torch.empty_like(dI)
        s = torch.cuda.current_stream()
        F.fmmfft_aggregate(h, dP, dI, dA, nb, nrhs, s)
        F.fmmfft_translate(h, dA, dB, nrhs, s)
        F.fmmfft_disaggregate(h, dP, dB, dy, nb, nrhs, s)
        torch.cuda.synchronize()
        assert F.fmmfft_poll_status(h) == 0
        plan = pl.Plan(K=K, L=L)
        ops = pl.operators(plan)
        ref = ff.disaggregate(P, w, pl.translate_with(lambda p: ops[p], ff.aggregate(P, I)))
        assert _rel(dy.cpu().numpy(), ref) <= (1e-10 if c128 else tol + 1e-5)
    finally:
        F.fmmfft_plan_destroy(h)


def test_far_field_argument_errors(native, cuda):
    F, torch = native, cuda
    K = (4, 4, 4)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, 1, 0, 0, 0.0)
    try:
        nd = F.fmmfft_plan_stats(h)["n_dir"]
        P = torch.zeros((nd, 2, 49, 4, 4, 4), dtype=torch.complex64, device="cuda")
        I = torch.zeros((1, 49, 4, 4, 4), dtype=torch.complex64, device="cuda")
        A = torch.zeros((nd, 2, 1, 4, 4, 4), dtype=torch.complex64, device="cuda")
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_aggregate(h, P, I, A, 49, 1)
        assert e.value.status == F.FMMFFT_ERR_UNSUPPORTED
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_aggregate(h, P, I, P, 2, 1)          # output overlaps the patterns
        assert e.value.status == F.FMMFFT_ERR_INVALID_ARG
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_disaggregate(h, P, A, I, 2, 0)
        assert e.value.status == F.FMMFFT_ERR_INVALID_ARG
    finally:
        F.fmmfft_plan_destroy(h)


def test_single_direction_and_many_rhs(native, cuda):
    """Degenerate grid: L = 0 with N_phi = 2L + 1 gives one direction (three of
    the four direction quarters of the disaggregation cluster are empty); 37
    right-hand sides exercise the RHS tiles' ragged tail.  The chain against
    the oracle's."""
    F, torch = native, cuda
    K, L, nb, nrhs = (5, 6, 7), 0, 3, 37
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, 0, 0, 0.0)
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_NPHI_RULE, 1)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, F.FMMFFT_PREC_C128)
        F.fmmfft_compress(h)
        assert F.fmmfft_plan_stats(h)["n_dir"] == 1
        _, w = F.fmmfft_plan_directions(h)
        box = (K[2], K[1], K[0])
        P = _cg(61, (1, 2, nb) + box)
        I = _cg(62, (nrhs, nb) + box)
        dP, dI = _dev(torch, P, True), _dev(torch, I, True)
        dA = torch.empty((1, 2, nrhs) + box, dtype=dP.dtype, device="cuda")
        dB, dy = torch.empty_like(dA), torch.empty_like(dI)
        s = torch.cuda.current_stream()
        F.fmmfft_aggregate(h, dP, dI, dA, nb, nrhs, s)
        F.fmmfft_translate(h, dA, dB, nrhs, s)
        F.fmmfft_disaggregate(h, dP, dB, dy, nb, nrhs, s)
        torch.cuda.synchronize()
        plan = pl.Plan(K=K, L=L, nphi_rule="paper")
        ops = pl.operators(plan)
        ref = ff.disaggregate(P, w, pl.translate_with(lambda p: ops[p], ff.aggregate(P, I)))
        assert _rel(dy.cpu().numpy(), ref) <= 1e-10
    finally:
        F.fmmfft_plan_destroy(h)
