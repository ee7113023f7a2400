"""Host-side pieces of bench.py (no GPU): the throughput units, the nominal
flop models of the roofline, the peaks, the workload table and the reference
arm.

The FP32 flop model is checked against a line-by-line count of the transforms
the yz pass performs: per field and x-slab, Kz forward and Kz inverse y-DFTs
of length n2 (5 n log2 n each), n2 z-lines of a forward and an inverse
n3-DFT and the n3-point Hadamard product (6 flops per complex product).  The
restores' complex MACs (tensor cores) are counted apart from it."""
import math

import pytest

import bench


def test_units_count_padded_voxels_directions_and_fields():
    assert bench._units((64, 64, 64), 162, 4) == 64 ** 3 * 162 * 8
    # the headline: Gvoxel.dir/s = units / t / 1e9
    assert bench._units((64, 64, 64), 162, 4) / 2.0e-3 / 1e9 == pytest.approx(169.87, rel=1e-4)


def _count(K, n, n_dir, nrhs):
    Kx, Ky, Kz = K
    n1, n2, n3 = n
    dft = lambda m: 5 * m * math.log2(m)
    total = 0.0
    for _ in range(n1 * n_dir):                     # (x, p) blocks
        for _ in range(2 * nrhs):                   # fields of the direction
            total += Kz * dft(n2) + Kz * dft(n2)   # forward and inverse y lines
            total += n2 * (dft(n3) + dft(n3) + 6 * n3)
    return total


@pytest.mark.parametrize("K,n,n_dir,nrhs", [((4, 4, 4), (8, 8, 8), 6, 1), ((3, 5, 6), (8, 16, 16), 4, 2),
                                            ((128, 128, 32), (256, 256, 64), 98, 16)])
def test_yz_flop_model_matches_a_line_count(K, n, n_dir, nrhs):
    assert bench.yz_fft_flops(K, n, n_dir, nrhs) == pytest.approx(_count(K, n, n_dir, nrhs), rel=1e-12)


def test_step_flops_add_the_x_passes():
    K, n, nd, nr = (6, 5, 7), (16, 16, 16), 4, 2
    x = nd * 2 * nr * 2 * K[1] * K[2] * 5 * n[0] * math.log2(n[0])
    assert bench.step_fp32_flops(K, n, nd, nr) == pytest.approx(x + bench.yz_fft_flops(K, n, nd, nr))


def test_restore_mac_counts():
    # slab: per (x, p) block (rb x n2) = (rb x ra)(ra x n2), then (n3 x rb)(rb x n2)
    n = (4, 8, 16)
    assert bench.slab_restore_macs(n, [(3, 5), (0, 7)]) == 4 * ((8 * 3 * 5 + 16 * 8 * 5) + 16 * 8 * 7)
    # Tucker-3D pre-pass H_p = U1 (n1 x r1) . C_p (r1 x r2 r3)
    assert bench.prepass_macs(n, 2, 3, 1, [(2, 3, 4), (1, 1, 1)]) == 4 * 2 * 12 + 4 * 1 * 1
    # TT-4D: T1 = U1 . C1 (n1 x r1)(r1 x n2 r2), R = U3 . C2 (n_dir x r3)(r3 x n3 r2)
    assert bench.prepass_macs(n, 5, 4, 2, [2, 3, 4]) == 4 * 2 * 8 * 3 + 5 * 4 * 16 * 3


def test_peaks():
    # FP32: 128 FMA lanes per SM at 2 flops per FMA
    assert bench.fp32_peak_tflops(152, 2070.0) == pytest.approx(80.54784)
    bf, _ = bench.tensor_peak_tflops({"bf16_tflops": 1800.0}, "bf16x3")
    tf, _ = bench.tensor_peak_tflops({"bf16_tflops": 1800.0}, "tf32")
    assert bf == 1800.0 and tf == pytest.approx(880.0)


def test_workload_table():
    W = bench.WORKLOADS
    assert bench.DEFAULT_WL in W
    d = W[bench.DEFAULT_WL]
    # the largest tolerance-1e-4 workload: the elongated 128 x 128 x 32 grid
    assert d["K"] == (128, 128, 32) and d["L"] == 6 and d["nrhs"] == 16 and d["tol"] == 1e-4
    assert bench.grid_of(bench.workload(bench.DEFAULT_WL)) == (256, 256, 64)
    assert bench.n_dir_of(d) == 98
    for name, w in W.items():
        assert (w["fmt"] == 0) == (w["dec"] == 0), name
        assert 1 <= w["fpd"] <= 2 * w["nrhs"], name


def test_sample_directions_spread_and_distinct():
    assert bench.sample_directions(98, 16) == sorted(set(bench.sample_directions(98, 16)))
    assert bench.sample_directions(98, 16)[0] == 0 and bench.sample_directions(98, 16)[-1] == 97
    assert bench.sample_directions(5, 16) == [0, 1, 2, 3, 4]


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


SMALL = "tucker3d_32cube_L8_tol1e-4_2pol_4rhs"


def test_reference_arm_prints_one_line_with_the_contract_keys():
    """bench.py --impl reference times the FP64 oracle on the host cores (one
    field per core and step, every core on its own direction) and prints one
    JSON line in the same metric and unit as the GPU arm, with its
    CPU-baseline and end-to-end objects (no host-device copies)."""
    out = _bench(["--impl", "reference", "--steps", "2", "--warmup", "1", "--workload", SMALL])
    assert len(out) == 1
    line = out[0]
    assert line["impl"] == "reference" and "unavailable" not in line
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and line["config"]["workload"] == SMALL
    cb = line["cpu_baseline"]
    cores = min(bench.host_cores(), 162)
    assert cb["kind"] == "oracle" and cb["cores"] == cores and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # the metric's units: a step translates one field (64^3 padded voxels of
    # one direction) per core
    assert math.isclose(line["value"], cores * 64 ** 3 / (line["ms_per_step"] * 1e-3) / 1e9, rel_tol=1e-9)


def test_cpu_baseline_sample_and_its_accuracy_reference(tmp_path):
    """The CPU baseline runs the oracle on one sampled direction per host core
    and, for the accuracy check, saves the oracle's compressed translations
    and the uncompressed FP64 ones of the same fields: on the 32^3 workload
    their difference is the Tucker-3D compression error, within tol."""
    import numpy as np
    cb = bench.run_cpu_baseline(SMALL, str(tmp_path / "o.npz"))
    assert cb["value"] > 0 and cb["cores"] == min(bench.host_cores(), 162) and cb["kind"] == "oracle"
    d = np.load(tmp_path / "o.npz")
    assert d["exact"].shape == (cb["cores"], 8, 32, 32, 32)
    err = np.linalg.norm(d["oracle"] - d["exact"]) / np.linalg.norm(d["exact"])
    assert 0 < err <= 1e-4


def test_reference_arm_runs_on_rank_zero_only():
    assert _bench(["--impl", "reference", "--steps", "1", "--warmup", "1", "--workload", SMALL],
                  {"RANK": "1"}) == []
