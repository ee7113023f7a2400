"""Pin of the oracle's translation on a partly occupied box grid (Sec. II.A:
boxes without basis functions have A_v = 0 and need no translated field).

The FFT route with the occupancy mask must equal the definition written out:
B(v') = sum over occupied v of T(v' - v) A(v) at occupied v', zero at empty
v' -- the brute-force Toeplitz sum restricted to occupied boxes, on tiny
grids (a sphere-like shell and a random mask).  A full mask reduces to the
unmasked translation exactly."""
import numpy as np
import pytest

from oracle import operator as op
from oracle import pipeline as pl
from oracle import translate as tr
from seeded_inputs import field_spectra, shell_occupancy as shell_mask


@pytest.mark.parametrize("K,kind", [((5, 4, 6), "shell"), ((4, 5, 3), "random"), ((6, 6, 6), "shell")])
def test_masked_translation_is_the_restricted_direct_sum(K, kind):
    plan = pl.Plan(K=K, L=2)
    kh = plan.directions()
    rng = np.random.default_rng(5)
    m = shell_mask(K) if kind == "shell" else rng.random((K[2], K[1], K[0])) < 0.5
    assert 0 < m.sum() < m.size
    S = field_spectra(11, plan.n_dir, 1, K)
    p = 3
    That = pl.operators(plan, [p])[0]
    got = pl.translate_occupied(lambda q: That, S[p:p + 1], m)[0, 0, 0]
    Kx, Ky, Kz = K
    d = [np.arange(-(k - 1), k) for k in K]
    DX, DY, DZ = np.meshgrid(*d, indexing="ij")
    Tgrid = op.operator_at(kh[p], DX, DY, DZ, plan.a, plan.k0, plan.L, plan.near_rule, plan.prefactor,
                           plan.kappa, plan.eps_r)
    want = np.where(m, tr.translate_field_direct(Tgrid, np.where(m, S[p, 0, 0], 0)), 0)
    np.testing.assert_allclose(got, want, atol=1e-12 * np.abs(want).max())
    assert np.all(got[~m] == 0)


def test_full_mask_is_the_plain_translation():
    K = (4, 5, 3)
    plan = pl.Plan(K=K, L=1)
    ops = pl.operators(plan)
    S = field_spectra(12, plan.n_dir, 2, K)
    full = np.ones((K[2], K[1], K[0]), bool)
    assert np.array_equal(pl.translate_occupied(lambda q: ops[q], S, full), pl.translate_with(lambda q: ops[q], S))
