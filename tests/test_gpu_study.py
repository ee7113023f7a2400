"""Compression study with GPU timings (Sec. III.A): one small case translated
with its compressed and its plain operator."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_study_case_times_compressed_and_plain(native, cuda):
    from paper_2010_00520_gb300 import study as S
    c = S.StudyCase(fmt="tucker3d", K=8, L=4, tol=1e-4, eps_r=2 - 1j)
    row = S.gpu_case(c, S.host_case(c), nrhs=1, steps=5, warmup=3)
    g = row.gpu
    assert g["ms_compressed"] > 0 and g["ms_plain"] > 0
    assert math.isfinite(g["overhead"]) and g["overhead"] > -1
    assert "ms compressed" in S.table([row])
