"""Compression study (Sec. III.A) through the library's host set-up.

* Table II, printed ranks at n = 32 (the 8-lambda sphere: K = 16 boxes of
  0.5 lambda, L = 14, 435 directions, gamma = 1e-6): the direction-mode ranks
  of the 4D formats are exactly the printed 225 = (L+1)^2; the spatial ranks of
  the 3D formats depend on the near-field rule (reading T): the printed
  kappa = 4 rule gives 31, the Chebyshev shell 27, and near offsets |d|^2 <= 5
  give Table II's 29;
* Table IV / Fig. 9: the memory saving grows and the ranks fall as the loss of
  the medium grows;
* the study rows agree with the library's own statistics.
"""
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table2_ranks.txt")


def _table2():
    out = {}
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            f, r, *vals = line.split()
            out[(f, r)] = dict(zip((32, 64, 128, 256), map(int, vals)))
    return out


@pytest.fixture(scope="module")
def study(native):
    from paper_2010_00520_gb300 import study as S
    return S


def test_sweep_builders(study):
    c = study.structure_size(["tucker3d"], diameters=(8, 16, 64))
    assert [x.K for x in c] == [16, 32, 128]
    c = study.box_size(["htucker"], sizes=(0.25, 0.5, 1.0), diameter=32)
    assert [(x.K, x.a) for x in c] == [(128, 0.25), (64, 0.5), (32, 1.0)]
    c = study.loss(["tt3d"], diameter=8)
    assert [x.multipoles() for x in c] == [18, 18, 20, 28]          # 703, 703, 861, 1653 directions
    c = study.accuracy(["tt3d"], digits=(3, 6), diameter=8)
    assert [(x.multipoles() + 1) * (2 * x.multipoles() + 1) for x in c] == [325, 496]


@pytest.mark.parametrize("fmt,rank", [("tucker4d", "r4"), ("tt4d", "r3")])
def test_table2_direction_rank(study, fmt, rank):
    row = study.host_case(study.StudyCase(fmt=fmt, K=16))
    assert row.n_dir == 435 and row.L == 14 and row.n == [32, 32, 32]
    r = row.ranks[3] if fmt == "tucker4d" else row.ranks[2]
    assert r == _table2()[(fmt, rank)][32] == (row.L + 1) ** 2


def test_table2_spatial_ranks_and_near_rule(study):
    t2 = _table2()
    printed = study.host_case(study.StudyCase(fmt="tucker3d", K=16))
    assert abs(max(printed.ranks) - t2[("tucker3d", "rmax")][32]) <= 3
    cheb = study.host_case(study.StudyCase(fmt="tucker3d", K=16, near_rule=0))
    shell5 = study.host_case(study.StudyCase(fmt="tucker3d", K=16, kappa=2.7))
    assert max(cheb.ranks) < t2[("tucker3d", "rmax")][32] < max(printed.ranks)
    assert max(shell5.ranks) == t2[("tucker3d", "rmax")][32]
    tt = study.host_case(study.StudyCase(fmt="tt3d", K=16, kappa=2.7))
    assert abs(max(tt.ranks) - t2[("tt3d", "rmax")][32]) <= 1


def test_loss_raises_memory_saving(study):
    rows = study.run(study.loss(["tucker3d"], diameter=8))
    sav = [r.saving for r in rows]
    rk = [max(r.ranks) for r in rows]
    assert sav[3] > sav[2] > sav[0] and sav[0] >= 0
    assert rk[3] < rk[0] and all(a >= b for a, b in zip(rk, rk[1:]))


def test_study_row_matches_library_statistics(study, native):
    c = study.StudyCase(fmt="htucker", K=4, L=3, tol=1e-4, near_rule=0, nphi_rule=0)
    row = study.host_case(c)
    h = native.fmmfft_plan_create(4, 4, 4, 0.5, 2 * np.pi, 3, 4, 3, 1e-4)
    try:
        r, _ = native.fmmfft_compress_host(h, restored=False)
        st = native.fmmfft_plan_stats(h)
        assert row.ranks == [int(v) for v in r]
        assert row.saving == st["saving"] and row.elements_compressed == st["elements_compressed"]
        assert row.n_dir == 32
    finally:
        native.fmmfft_plan_destroy(h)
    assert "| htucker | 4 |" in study.table([row])


def test_study_command_line_writes_rows(study, tmp_path, capsys):
    """`python -m paper_2010_00520_gb300.study`: a host-only sweep of the
    structure size (a 1-lambda sphere: 2 x 2 x 2 boxes of 0.5 lambda) writes
    one row per case, as JSON lines, a table and a JSON file."""
    import json
    out = tmp_path / "rows.json"
    study.main(["size", "--diameters", "1", "1.5", "--formats", "tucker3d", "tt3d", "--tol", "1e-4",
                "--json", str(out)])
    rows = json.loads(out.read_text())
    assert [r["case"]["fmt"] for r in rows] == ["tucker3d", "tt3d", "tucker3d", "tt3d"]
    assert [r["case"]["K"] for r in rows] == [2, 2, 3, 3]
    assert all(r["n_dir"] == 435 and r["L"] == 14 for r in rows)
    assert all(0.0 <= r["saving"] < 1.0 and r["gpu"] == {} for r in rows)
    printed = capsys.readouterr().out
    assert printed.count('{"case"') == 4 and "| tucker3d | 2 |" in printed


def test_study_reports_the_restore_error_on_request(study, tmp_path):
    """--restore-error: each row carries the FP64 relative error of the stored
    operator against the uncompressed one, within the case's tolerance for
    every format; without it the field stays -1 and the table has no column."""
    import json
    rows = study.run([study.StudyCase(fmt=f, K=4, L=3, tol=1e-4, near_rule=0, nphi_rule=0)
                      for f in ("tucker3d", "tt3d", "tucker4d", "htucker", "tt4d")], restore_error=True)
    assert all(0.0 < r.restore_rel_err <= 1e-4 for r in rows), [r.restore_rel_err for r in rows]
    assert "FP64 restore error" in study.table(rows)
    plain = study.host_case(study.StudyCase(fmt="tucker3d", K=4, L=3, tol=1e-4, near_rule=0, nphi_rule=0))
    assert plain.restore_rel_err == -1.0 and "FP64 restore error" not in study.table([plain])
    out = tmp_path / "rows.json"
    study.main(["size", "--diameters", "2", "--formats", "tucker3d", "--tol", "1e-4", "--restore-error",
                "--json", str(out)])
    (row,) = json.loads(out.read_text())
    assert 0.0 < row["restore_rel_err"] <= 1e-4
