"""Host-side pieces of bench.py (no GPU): the throughput units, the nominal
flop model of the yz roofline and the workload table.

The flop model is checked against a line-by-line count of the transforms the
yz pass performs: per field and x-slab, Kz forward and Kz inverse y-DFTs of
length n2 (5 n log2 n each), n2 z-lines of a forward and an inverse n3-DFT
and the n3-point Hadamard product (6 flops per complex product), plus the
complex MACs of the slab restore (8 flops each)."""
import math

import pytest

import bench


def test_units_count_padded_voxels_directions_and_fields():
    assert bench._units((64, 64, 64), 162, 4) == 64 ** 3 * 162 * 8
    # the headline: Gvoxel.dir/s = units / t / 1e9
    assert bench._units((64, 64, 64), 162, 4) / 2.0e-3 / 1e9 == pytest.approx(169.87, rel=1e-4)


def _count(K, n, n_dir, nrhs, ranks=None):
    Kx, Ky, Kz = K
    n1, n2, n3 = n
    dft = lambda m: 5 * m * math.log2(m)
    total = 0.0
    for _ in range(n1 * n_dir):                     # (x, p) blocks
        for _ in range(2 * nrhs):                   # fields of the direction
            total += Kz * dft(n2) + Kz * dft(n2)   # forward and inverse y lines
            total += n2 * (dft(n3) + dft(n3) + 6 * n3)
    if ranks:
        for ra, rb in ranks:
            total += n1 * 8 * (n2 * ra * rb + n3 * n2 * rb)
    return total


@pytest.mark.parametrize("K,n,n_dir,nrhs,ranks", [((4, 4, 4), (8, 8, 8), 6, 1, None),
                                                  ((3, 5, 6), (8, 16, 16), 4, 2, [(3, 5)] * 4),
                                                  ((6, 6, 6), (16, 16, 16), 3, 1, [(0, 7), (0, 9), (0, 4)])])
def test_yz_flop_model_matches_a_line_count(K, n, n_dir, nrhs, ranks):
    assert bench.yz_flops(K, n, n_dir, nrhs, ranks) == pytest.approx(_count(K, n, n_dir, nrhs, ranks), rel=1e-12)


def test_step_flops_add_the_x_passes():
    K, n, nd, nr = (6, 5, 7), (16, 16, 16), 4, 2
    x = nd * 2 * nr * 2 * K[1] * K[2] * 5 * n[0] * math.log2(n[0])
    assert bench.step_flops(K, n, nd, nr) == pytest.approx(x + bench.yz_flops(K, n, nd, nr))


def test_workload_table():
    W = bench.WORKLOADS
    assert bench.DEFAULT_WL in W
    d = W[bench.DEFAULT_WL]
    assert d["K"] == (32, 32, 32) and d["L"] == 8 and d["nrhs"] == 4 and d["tol"] == 1e-4
    for name, w in W.items():
        assert (w["fmt"] == 0) == (w["dec"] == 0), name
        assert 2 * (w["L"] + 1) ** 2 >= 1


def _bench(args, env_extra=None):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, cwd=root, env=env,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return [json.loads(l) for l in lines]


def test_reference_arm_prints_one_line_with_the_contract_keys():
    """bench.py --impl reference times the FP64 oracle on the host (one field
    of the benchmark workload per step) and prints one JSON line in the same
    metric and unit as the GPU arm, with its CPU-baseline and end-to-end
    objects (no host-device copies)."""
    out = _bench(["--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert len(out) == 1
    line = out[0]
    assert line["impl"] == "reference" and "unavailable" not in line
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and line["config"]["workload"] == bench.WL["name"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # the metric's units: one field is 64^3 padded voxels of one direction
    assert math.isclose(line["value"], 64 ** 3 / (line["ms_per_step"] * 1e-3) / 1e9, rel_tol=1e-9)


def test_reference_arm_runs_on_rank_zero_only():
    assert _bench(["--impl", "reference", "--steps", "1", "--warmup", "1"], {"RANK": "1"}) == []
