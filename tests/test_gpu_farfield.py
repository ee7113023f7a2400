"""GPU parity of the far-field steps (Eqs. 4 and 6) against the oracle.

Random patterns, coefficients and spectra (seeded complex Gaussians), ragged
box counts (not multiples of the 128-box tiles), basis-function and RHS counts
off the kernels' tile sizes, odd direction counts.  Bounds: complex64 rel L2
2e-6 for aggregation (sums of nb FP32 products), 1e-5 for disaggregation (sums
of 2 n_dir products, sqrt(2 n_dir) eps growth); complex128 1e-12.  The chain
aggregate -> translate -> disaggregate, and the fused translate +
disaggregate, are checked against the oracle's chain.  Every oracle input
comes from the oracle or the seeded generator: the quadrature weights are the
oracle's own direction grid (Sec. II.A), not the library's.
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


def _w(L, nphi):
    """The oracle's quadrature weights of the plan's direction grid."""
    return dr.direction_grid(L, "paper" if nphi == 1 else "benchmark")[1]


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
        w = _w(L, nphi)
        assert len(w) == nd
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
        w = _w(L, 0)
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
        w = _w(L, 1)
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


@pytest.mark.parametrize("K,L,nphi,nb,nrhs,fmt,dec,prec", [
    ((5, 7, 3), 2, 1, 3, 5, 0, 0, 0),        # ragged boxes, odd RHS count, complex128
    ((8, 8, 8), 3, 0, 16, 4, 0, 0, 1),       # plain complex64
    ((10, 8, 12), 3, 0, 20, 3, 3, 1, 2),     # Tucker-3D 3xTF32, two basis-function chunks
    ((16, 12, 10), 4, 1, 5, 2, 4, 3, 1),     # H-Tucker, FP32 restores
    ((33, 6, 4), 2, 0, 7, 1, 0, 0, 1),       # Kx = 33: tiles of three rows (99 boxes), n1 = 128
    ((5, 6, 7), 0, 1, 3, 6, 0, 0, 0),        # one direction: three empty direction quarters
])
def test_translate_disaggregate_matches_oracle(native, cuda, K, L, nphi, nb, nrhs, fmt, dec, prec):
    """fmmfft_translate_disaggregate (Eq. 5 then Eq. 6, the translated fields
    kept on chip) against the oracle's translation followed by its
    disaggregation on the same inputs; and against the library's unfused
    chain (translate, then disaggregate) to rounding."""
    F, torch = native, cuda
    tol = 1e-4
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, fmt, dec, tol if fmt else 0.0)
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_NPHI_RULE, nphi)
        F.fmmfft_compress(h)
        c128 = prec == 0
        nd = F.fmmfft_plan_stats(h)["n_dir"]
        w = _w(L, nphi)
        assert len(w) == nd
        box = (K[2], K[1], K[0])
        P = _cg(71 + nb, (nd, 2, nb) + box)
        S = _cg(72 + nrhs, (nd, 2, nrhs) + box)
        dP, dS = _dev(torch, P, c128), _dev(torch, S, c128)
        dy = torch.full((nrhs, nb) + box, float("nan"), dtype=dP.dtype, device="cuda")
        dB = torch.empty_like(dS)
        dy2 = torch.empty_like(dy)
        s = torch.cuda.current_stream()
        F.fmmfft_translate_disaggregate(h, dS, dP, dy, nb, nrhs, s)
        F.fmmfft_translate(h, dS, dB, nrhs, s)
        F.fmmfft_disaggregate(h, dP, dB, dy2, nb, nrhs, s)
        torch.cuda.synchronize()
        assert F.fmmfft_poll_status(h) == 0
        y, y2 = dy.cpu().numpy(), dy2.cpu().numpy()
        assert np.isfinite(y).all()
        plan = pl.Plan(K=K, L=L, nphi_rule="paper" if nphi == 1 else "benchmark")
        ops = pl.operators(plan)
        Sd = S.astype(np.complex128 if c128 else np.complex64).astype(np.complex128)
        Pd = P.astype(np.complex128 if c128 else np.complex64).astype(np.complex128)
        ref = ff.disaggregate(Pd, w, pl.translate_with(lambda p: ops[p], Sd))
        bound = 1e-10 if c128 else (tol + 1e-5 if fmt else 1e-5)
        assert _rel(y, ref) <= bound
        assert _rel(y, y2) <= (1e-12 if c128 else 1e-5)
    finally:
        F.fmmfft_plan_destroy(h)


def test_translate_disaggregate_argument_errors(native, cuda):
    F, torch = native, cuda
    K = (4, 4, 4)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, 1, 0, 0, 0.0)
    try:
        nd = F.fmmfft_plan_stats(h)["n_dir"]
        P = torch.zeros((nd, 2, 2, 4, 4, 4), dtype=torch.complex64, device="cuda")
        S = torch.zeros((nd, 2, 1, 4, 4, 4), dtype=torch.complex64, device="cuda")
        y = torch.zeros((1, 2, 4, 4, 4), dtype=torch.complex64, device="cuda")
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_translate_disaggregate(h, S, P, y, 2, 1)       # no operator yet
        assert e.value.status == F.FMMFFT_ERR_NOT_COMPRESSED
        F.fmmfft_compress(h)
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_translate_disaggregate(h, S, P, P, 2, 1)       # output overlaps the patterns
        assert e.value.status == F.FMMFFT_ERR_INVALID_ARG
    finally:
        F.fmmfft_plan_destroy(h)
