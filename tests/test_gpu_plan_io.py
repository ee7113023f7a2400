"""GPU checks of plan files: a compressed plan saved and loaded back restores
and translates bit-identically to the original (same factors, same schedule),
without repeating the FP64 set-up; a plain plan is regenerated on load."""
import numpy as np
import pytest

from seeded_inputs import field_spectra

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


@pytest.mark.parametrize("fmt,dec,tol,prec", [(3, 1, 1e-4, 2), (4, 3, 1e-4, 2), (4, 2, 1e-4, 1), (3, 2, 1e-4, 1),
                                              (0, 0, 0.0, 1)])
def test_saved_plan_translates_identically(native, cuda, tmp_path, fmt, dec, tol, prec):
    F, torch = native, cuda
    K, L, nrhs = (7, 6, 9), 3, 2
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, fmt, dec, tol)
    h2 = None
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
        F.fmmfft_compress(h)
        path = str(tmp_path / "p.plan")
        F.fmmfft_plan_save(h, path)
        h2 = F.fmmfft_plan_load(path)
        a, b = F.fmmfft_plan_stats(h), F.fmmfft_plan_stats(h2)
        for k in ("n_dir", "n", "format", "decomp", "precision", "max_rank", "elements_compressed",
                  "restore_on_tensor_cores"):
            assert a[k] == b[k], k
        S = field_spectra(77, a["n_dir"], nrhs, K).astype(np.complex64)
        x = torch.from_numpy(S).to("cuda")
        y1, y2 = torch.empty_like(x), torch.empty_like(x)
        F.fmmfft_translate(h, x, y1, nrhs)
        F.fmmfft_translate(h2, x, y2, nrhs)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
    finally:
        F.fmmfft_plan_destroy(h)
        if h2:
            F.fmmfft_plan_destroy(h2)


@pytest.mark.parametrize("fmt,dec,tol", [(3, 1, 1e-4), (0, 0, 0.0)])
def test_saved_shard_plan_in_a_lossy_medium(native, cuda, tmp_path, fmt, dec, tol):
    """The options a plan file carries beyond the first version: the medium's
    permittivity and the direction block of a shard plan (a plain plan is
    regenerated on load from them)."""
    F, torch = native, cuda
    K, L, nrhs = (7, 6, 9), 3, 1
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, fmt, dec, tol)
    h2 = None
    try:
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_EPS_R_RE, 2.0)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_EPS_R_IM, -1.0)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_DIR_FIRST, 9)
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_DIR_COUNT, 13)
        F.fmmfft_compress(h)
        path = str(tmp_path / "s.plan")
        F.fmmfft_plan_save(h, path)
        h2 = F.fmmfft_plan_load(path)
        assert F.fmmfft_plan_stats(h2)["n_dir"] == 13
        k1, w1 = F.fmmfft_plan_directions(h)
        k2, w2 = F.fmmfft_plan_directions(h2)
        assert np.array_equal(k1, k2) and np.array_equal(w1, w2)
        S = field_spectra(78, 13, nrhs, K).astype(np.complex64)
        x = torch.from_numpy(S).to("cuda")
        y1, y2 = torch.empty_like(x), torch.empty_like(x)
        F.fmmfft_translate(h, x, y1, nrhs)
        F.fmmfft_translate(h2, x, y2, nrhs)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
    finally:
        F.fmmfft_plan_destroy(h)
        if h2:
            F.fmmfft_plan_destroy(h2)
