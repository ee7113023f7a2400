#!/usr/bin/env python
"""Throughput of the compressed FMM-FFT translation stage on GPUs of one node.

One step = one fmmfft_translate call: every field of the workload (all
directions, both polarisations, every RHS) translated through Eq. 5 with the
operator restored from its compressed store (Sec. II.C).  The uncompressed
(plain) translation of the same fields is timed beside it.

Workload (default): the elongated structure, 128 x 128 x 32 boxes of edge 0.5
wavelength (k0 = 2 pi), L = 6, 98 directions (Gauss-Legendre x 14 uniform
phi), FFT grid 256 x 256 x 64, Tucker-3D HOSVD at tol 1e-4 against the
uncompressed complex64 operator (3.3 GB), complex64 fields with FP32 FFTs and
3xTF32 tensor-core restores, 2 polarisations x 16 RHS of seeded i.i.d.
complex Gaussian box spectra (synthetic stand-ins for the aggregated fields of
a meshed structure).  `--workload` selects the others (32^3 boxes L = 8, the
64^3-box 4D formats, ...).

Metric: Gvoxel.dir/s = n1 n2 n3 * n_dir * 2 * nrhs / t / 1e9 (padded voxels
times fields translated per second).  Inputs and outputs (13 GB each on the
default workload) are larger than the 129 MB L2, so no flush is needed
between steps.

Launch: python bench.py [--gpus N --steps K --warmup W] (torchrun for N > 1:
by default the ranks split the directions of one problem, no collective on
the data path).  --impl reference times the FP64 CPU oracle on the host cores
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "translation Gvoxel·dir/s, compressed vs plain on one GB300, at rel err ≤1e-4"
UNIT = "Gvoxel·dir/s"
# Workloads (box edge 0.5 wavelength, k0 = 2 pi, seeded complex Gaussian fields).
# fmt / dec: FMMFFT_FORMAT_* / FMMFFT_DECOMP_* of the compressed arm (0 / 0: the
# workload has only the plain arm); c128: complex128 arithmetic; restore: the
# compressed arm's tensor-core arithmetic; fpd: fields per sampled direction of
# the CPU oracle (baseline and accuracy sample).
WORKLOADS = {
    "tucker3d_128x128x32_L6_tol1e-4_2pol_16rhs": dict(K=(128, 128, 32), L=6, tol=1e-4, nrhs=16, seed=1005,
                                                     fmt=3, dec=1, restore="3xtf32", fpd=2),
    "htucker4d_128x128x32_L6_tol1e-4_2pol_16rhs": dict(K=(128, 128, 32), L=6, tol=1e-4, nrhs=16, seed=1005,
                                                      fmt=4, dec=3, restore="3xtf32", fpd=2),
    "tucker3d_32cube_L8_tol1e-4_2pol_4rhs": dict(K=(32, 32, 32), L=8, tol=1e-4, nrhs=4, seed=1002, fmt=3, dec=1,
                                                restore="3xtf32", fpd=8),
    "plain_c128_8cube_L5_2pol_1rhs": dict(K=(8, 8, 8), L=5, tol=0.0, nrhs=1, seed=1001, fmt=0, dec=0, c128=True,
                                          fpd=2),
    "tt4d_64cube_L10_tol1e-3_2pol_1rhs": dict(K=(64, 64, 64), L=10, tol=1e-3, nrhs=1, seed=1003, fmt=4, dec=2,
                                             restore="bf16x3", fpd=2),
    "htucker4d_64cube_L10_tol1e-3_2pol_1rhs": dict(K=(64, 64, 64), L=10, tol=1e-3, nrhs=1, seed=1003, fmt=4,
                                                  dec=3, restore="bf16x3", fpd=2),
}
# the largest tol-1e-4 workload that fits one GPU
DEFAULT_WL = "tucker3d_128x128x32_L6_tol1e-4_2pol_16rhs"
FORMAT_NAMES = {(3, 1): "tucker3d", (3, 2): "tt3d", (4, 1): "tucker4d", (4, 2): "tt4d", (4, 3): "htucker4d",
                (0, 0): "none"}
FAR_NB = 16                  # basis functions per box of the far-field steps (Eqs. 4, 6)
# version of each yz kernel's code the committed DRAM-traffic figures were
# taken on (a figure counts only while its kernel is unchanged)
YZ_KERNEL_VERSION = {"yz_kernel": 6, "yzl_kernel": 7}


def workload(name: str) -> dict:
    return dict(WORKLOADS[name], name=name, a=0.5, k0=2 * math.pi)


def embed_extent(k: int) -> int:
    n = 1
    while n < 2 * k - 1:
        n *= 2
    return max(n, 2)


def grid_of(W) -> tuple:
    return tuple(embed_extent(k) for k in W["K"])


def n_dir_of(W) -> int:
    return 2 * (W["L"] + 1) ** 2


def _units(n, n_dir, nrhs):
    return n[0] * n[1] * n[2] * n_dir * 2 * nrhs


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# The FP64 oracle on the host cores: one spawned process per sampled
# direction, one BLAS thread each.  Used by the CPU baseline (with the
# accuracy sample) and by the reference arm.
# ---------------------------------------------------------------------------
def oracle_mode(W) -> str:
    """What the oracle runs per field: the Tucker-3D restore of the field's
    direction (Fig. 3(a)) and Eq. 5, or for the other formats Eq. 5 with the
    uncompressed FP64 operator (the oracle's decomposition of a whole 4D
    operator of these sizes takes far longer than a bench run)."""
    return "tucker3d" if (W["fmt"], W["dec"]) == (3, 1) else "plain"


def sample_directions(n_dir: int, count: int) -> list:
    count = max(1, min(count, n_dir))
    return [int(round(i * (n_dir - 1) / max(count - 1, 1))) for i in range(count)]


def _oracle_worker(wl_name, p, fields_per_step, steps, want_exact, barrier, queue):
    """One sampled direction p.  Untimed: the operator (Eq. 7, embedding,
    FFT), its HOSVD (Tucker-3D workloads) and the fields.  Timed, per step
    after a barrier: the restore of T~_p (Tucker-3D) and Eq. 5 for the step's
    fields.  Untimed afterwards: the same fields through the uncompressed
    operator when `want_exact`.  Fields are rounded to complex64 as the GPU
    receives them."""
    import numpy as np
    from oracle import decomp as D
    from oracle import pipeline as pl
    from oracle import translate as tr
    from seeded_inputs import field_spectra_rows

    try:
        W = workload(wl_name)
        K, nrhs, nf = W["K"], W["nrhs"], 2 * W["nrhs"]
        plan = pl.Plan(K=K, L=W["L"])
        op = pl.operators(plan, [p])[0]
        mode = oracle_mode(W)
        tk = D.tucker_hosvd(op, W["tol"]) if mode == "tucker3d" else None
        js = [[(s * fields_per_step + i) % nf for i in range(fields_per_step)] for s in range(steps)]
        flat = sorted({j for step in js for j in step})
        A = dict(zip(flat, field_spectra_rows(W["seed"], plan.n_dir, nrhs, K, np.array(flat) + p * nf)
                     .astype(np.complex64).astype(np.complex128)))
        times, outs = [], {}
        for step in js:
            barrier.wait(timeout=3600)
            t0 = time.perf_counter()
            Th = D.tucker3d_restore_steps(tk.core, *tk.factors) if tk is not None else op
            for j in step:
                outs[j] = tr.translate_field_fft(Th, A[j])
            times.append((t0, time.perf_counter()))
        exact = {}
        if want_exact:
            for j in flat:
                exact[j] = outs[j] if tk is None else tr.translate_field_fft(op, A[j])
        queue.put({"p": p, "times": times, "fields": flat, "out": [outs[j] for j in flat],
                   "exact": [exact[j] for j in flat] if want_exact else None})
    except BaseException as e:          # report, then let the parent fail cleanly
        try:
            barrier.abort()
        except Exception:
            pass
        queue.put({"p": p, "error": repr(e)})


def run_oracle_pool(wl_name, dirs, fields_per_step, steps, want_exact, timeout_s=3600):
    """Runs _oracle_worker for every direction of `dirs` at once (spawned
    processes, one BLAS thread each).  Returns (results by direction, per-step
    wall seconds: last end minus first start over the workers)."""
    import multiprocessing as mp

    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(len(dirs))
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(wl_name, p, fields_per_step, steps, want_exact, barrier,
                                                      queue), daemon=True) for p in dirs]
    for pr in procs:
        pr.start()
    res = {}
    deadline = time.time() + timeout_s
    while len(res) < len(procs):
        r = queue.get(timeout=max(1.0, deadline - time.time()))
        if "error" in r:
            for pr in procs:
                pr.terminate()
            raise RuntimeError(f"oracle worker for direction {r['p']} failed: {r['error']}")
        res[r["p"]] = r
    for pr in procs:
        pr.join(timeout=60)
    step_s = [max(res[p]["times"][s][1] for p in dirs) - min(res[p]["times"][s][0] for p in dirs)
              for s in range(steps)]
    return res, step_s


def cpu_baseline_child(wl_name: str, out_path: str = ""):
    """The oracle on all host cores, one sampled direction per core, `fpd`
    fields of each (one step).  Prints the timing; with out_path saves the
    oracle's outputs and, for the accuracy check, the uncompressed FP64
    translations of the same fields (.npz)."""
    import numpy as np

    W = workload(wl_name)
    cores = host_cores()
    nd = n_dir_of(W)
    dirs = sample_directions(nd, cores)
    fpd = min(W["fpd"], 2 * W["nrhs"])
    res, step_s = run_oracle_pool(wl_name, dirs, fpd, 1, bool(out_path))
    n = grid_of(W)
    nfields = len(dirs) * fpd
    if out_path:
        np.savez(out_path, dirs=np.array(dirs), fields=np.array([res[p]["fields"] for p in dirs]),
                 oracle=np.stack([np.stack(res[p]["out"]) for p in dirs]),
                 exact=np.stack([np.stack(res[p]["exact"]) for p in dirs]))
    print(json.dumps({"seconds": step_s[0], "units": n[0] * n[1] * n[2] * nfields, "fields": nfields,
                      "dirs": len(dirs), "fpd": fpd, "cores": len(dirs)}))


def run_cpu_baseline(wl_name: str, out_path: str = ""):
    W = workload(wl_name)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-child", wl_name]
    if out_path:
        cmd += ["--cpu-baseline-out", out_path]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    what = ("Tucker-3D restore of the direction (Fig. 3(a)) + FFT translation (Eq. 5)"
            if oracle_mode(W) == "tucker3d" else "FFT translation (Eq. 5) with the uncompressed operator")
    return {"value": d["units"] / d["seconds"] / 1e9, "unit": UNIT, "cores": d["cores"], "kind": "oracle",
            "seconds": d["seconds"],
            "sample": f"{d['dirs']} of {n_dir_of(W)} directions x {d['fpd']} fields of the {wl_name} workload, "
                      f"one direction per host core ({d['cores']} processes, 1 thread each, run at once): "
                      f"{what}, FP64 NumPy; operator generation and decomposition untimed"}


# ---------------------------------------------------------------------------
# reference arm: the oracle as the reference implementation
# ---------------------------------------------------------------------------
def reference_child(wl_name: str, steps: int, warmup: int):
    """A step translates one field per host core with the oracle, every core
    on its own direction of the workload (restore of T~_p and Eq. 5 in FP64
    for Tucker-3D workloads); prints the per-step wall seconds."""
    W = workload(wl_name)
    cores = host_cores()
    dirs = sample_directions(n_dir_of(W), cores)
    _, step_s = run_oracle_pool(wl_name, dirs, 1, steps + warmup, False)
    print(json.dumps({"seconds": step_s[warmup:], "cores": len(dirs)}))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W = workload(args.workload)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--reference-child", args.workload,
                        str(args.steps), str(args.warmup)],
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, timeout=3600)
    if r.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + r.stderr[-300:]}))
        return
    d = json.loads(r.stdout.strip().splitlines()[-1])
    secs, cores = d["seconds"], d["cores"]
    n = grid_of(W)
    units = n[0] * n[1] * n[2] * cores
    val = units * len(secs) / sum(secs) / 1e9
    what = ("Tucker-3D restore + FFT translation" if oracle_mode(W) == "tucker3d"
            else "FFT translation with the uncompressed operator")
    sample = (f"{cores} fields per step, one per host core (each core on its own direction of the "
              f"{args.workload} workload, 1 thread); FP64 NumPy oracle ({what})")
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": config_of(W, W["nrhs"], 1, "host cores (no GPU)"),
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    out["config"]["step"] = f"{cores} fields of the workload per step, one per host core"
    print(json.dumps(out))


def config_of(W, nrhs, world, parallelism):
    return {"workload": W["name"] if nrhs == W["nrhs"] else W["name"].replace(f"{W['nrhs']}rhs", f"{nrhs}rhs"),
            "K": list(W["K"]), "n": list(grid_of(W)), "L": W["L"], "n_dir": n_dir_of(W), "nrhs": nrhs,
            "fields": n_dir_of(W) * 2 * nrhs,
            "format": FORMAT_NAMES[(W["fmt"], W["dec"])], "tol": W["tol"],
            "parallelism": parallelism or ("1 GPU" if world == 1 else f"{world} GPUs")}


# ---------------------------------------------------------------------------
# flop / byte models of one step (nominal 5 N log2 N flops per complex DFT)
# ---------------------------------------------------------------------------
def yz_fft_flops(K, n, n_dir, nrhs):
    """FP32 CUDA-core flops of one yz launch: per field and x-slab Kz forward
    and Kz inverse y-DFTs of length n2, n2 z-lines of a forward and an
    inverse n3-DFT and the n3-point Hadamard product (6 flops per point)."""
    Kx, Ky, Kz = K
    n1, n2, n3 = n
    per_field_slab = 2 * Kz * 5 * n2 * math.log2(n2) + n2 * (2 * 5 * n3 * math.log2(n3) + 6 * n3)
    return n1 * n_dir * 2 * nrhs * per_field_slab


def x_fft_flops(K, n, n_dir, nrhs):
    """Both x passes: a forward and an inverse n1-DFT per (y, z) row of every field."""
    Kx, Ky, Kz = K
    return n_dir * 2 * nrhs * 2 * Ky * Kz * 5 * n[0] * math.log2(n[0])


def step_fp32_flops(K, n, n_dir, nrhs):
    return x_fft_flops(K, n, n_dir, nrhs) + yz_fft_flops(K, n, n_dir, nrhs)


def slab_restore_macs(n, slab_ranks):
    """Complex MACs of the slab restores of one yz launch (per (x, p) block:
    (ra x n2 from ra x rb by n2 x ra) when ra > 0, then (n3 x rb)(rb x n2))."""
    n1, n2, n3 = n
    return n1 * sum(n2 * ra * rb + n3 * n2 * rb for (ra, rb) in slab_ranks)


def prepass_macs(n, n_dir, fmt, dec, ranks):
    """Complex MACs of the restore pre-pass and 4D core generation of one call.
    ranks: 3D formats, per direction (r1, r2, r3); 4D formats, the plan's
    largest ranks (r1, r2, r3, r4, r12, r34) (TT-4D: (r1, r2, r3))."""
    n1, n2, n3 = n
    if fmt == 3 and dec == 1:                   # H_p = U1 . C_p
        return sum(n1 * r1 * r2 * r3 for (r1, r2, r3) in ranks)
    if fmt == 3:                                # T1_p = U1 . C1_p
        return sum(n1 * r1 * n2 * r2 for (r1, r2, _) in ranks)
    if dec == 2:                                # T1 = U1 . C1 (shared), R = U3 . C2
        r1, r2, r3 = ranks[:3]
        return n1 * r1 * n2 * r2 + n_dir * r3 * n3 * r2
    r1, r2, r3, r4, r12, r34 = ranks[:6]
    h = n_dir * n1 * r1 * r2 * r3              # H_p = U1 . C_p
    if dec == 1:                                # C_all = U4 . C(4)
        return h + n_dir * r4 * r1 * r2 * r3
    return h + r1 * r2 * r12 * r34 + n_dir * r4 * r34 * r3 + n_dir * r1 * r2 * r34 * r3


def slab_ranks_of(F, h, fmt, dec, n_dir):
    st = F.fmmfft_plan_stats(h)
    r = st["max_rank"]
    if fmt == 3:
        pr = F.fmmfft_plan_ranks(h)
        return [(int(a[1]), int(a[2])) if dec == 1 else (0, int(a[1])) for a in pr], [tuple(int(v) for v in a)
                                                                                     for a in pr]
    if dec == 2:
        return [(0, int(r[1]))] * n_dir, [int(v) for v in r]
    return [(int(r[1]), int(r[2]))] * n_dir, [int(v) for v in r]


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 CUDA-core peak: 128 lanes per SM, one FMA (2 flops) per lane per clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def tensor_peak_tflops(peaks: dict, restore: str) -> tuple:
    """Dense tensor-core peak for the restore's operand type: the measured
    bf16 burst figure for bf16 operands (BF16x3), scaled by the nominal
    TF32 / BF16 ratio 1.1 / 2.25 for TF32 operands (3xTF32, TF32)."""
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    if restore == "bf16x3":
        return bf16, f"measured bf16 burst {bf16:.0f} TFLOP/s"
    return bf16 * 1.1 / 2.25, f"measured bf16 burst {bf16:.0f} TFLOP/s x nominal TF32/BF16 1.1/2.25"


# The batched workload: 64 independent FMM-FFT instances of uneven box grids
# (K_i drawn uniformly from 16..32 per axis, so FFT extents 32 or 64), L drawn
# from 4..10, Tucker-3D per direction at tol 1e-4 with 3xTF32 restores, 2
# polarisations x 8 RHS each, seeded fields per instance.
BATCH_WL = "batch64_tucker3d_K16-32_L4-10_tol1e-4_2pol_8rhs"
BATCH = dict(instances=64, K=(16, 32), L=(4, 10), tol=1e-4, nrhs=8, seed=1004)


def batch_specs():
    import numpy as np
    rng = np.random.default_rng(BATCH["seed"])
    out = []
    for i in range(BATCH["instances"]):
        K = tuple(int(k) for k in rng.integers(BATCH["K"][0], BATCH["K"][1] + 1, size=3))
        L = int(rng.integers(BATCH["L"][0], BATCH["L"][1] + 1))
        out.append((K, L, BATCH["seed"] * 1000 + i))
    return out


def run_batch(args):
    """One step = one fmmfft_batch_translate over all instances (graph
    replay after the first calls); the same batch with one launch sequence
    per instance (FMMFFT_BATCH_SEPARATE=1) is timed beside it."""
    import torch

    import paper_2010_00520_gb300 as F
    from seeded_inputs import field_spectra_torch

    torch.cuda.set_device(0)
    if not os.path.exists(F.LIB_PATH):
        from paper_2010_00520_gb300 import build as _b
        _b.build()
    specs = batch_specs()
    plans, xs, ys, nr, units = [], [], [], [], 0
    t0 = time.perf_counter()
    for (K, L, seed) in specs:
        h = F.fmmfft_plan_create(*K, 0.5, 2 * math.pi, L, 3, 1, BATCH["tol"])
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, F.FMMFFT_PREC_C64_3XTF32)
        F.fmmfft_compress(h)
        st = F.fmmfft_plan_stats(h)
        plans.append(h)
        xs.append(field_spectra_torch(seed, st["n_dir"], BATCH["nrhs"], K, device="cuda"))
        ys.append(torch.empty_like(xs[-1]))
        nr.append(BATCH["nrhs"])
        units += _units(st["n"], st["n_dir"], BATCH["nrhs"])
    t_setup = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    io_bytes = sum(2 * x.numel() * x.element_size() for x in xs)

    def timed(separate):
        os.environ["FMMFFT_BATCH_SEPARATE"] = "1" if separate else "0"
        b = F.fmmfft_batch_create(plans)
        try:
            for _ in range(max(args.warmup, 3)):
                F.fmmfft_batch_translate(b, xs, ys, nr, stream)
            stream.synchronize()
            shared = F.fmmfft_batch_shared_count(b)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
            ev[0].record(stream)
            for i in range(args.steps):
                F.fmmfft_batch_translate(b, xs, ys, nr, stream)
                ev[i + 1].record(stream)
            stream.synchronize()
            for h in plans:
                assert F.fmmfft_poll_status(h) == 0
            per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
            return ev[0].elapsed_time(ev[-1]) / args.steps, per, shared
        finally:
            F.fmmfft_batch_destroy(b)

    clocks = ClockSampler(0)
    clocks.start()
    ms, per, shared = timed(False)
    clk = clocks.stop()
    ms_sep, _, _ = timed(True)
    os.environ.pop("FMMFFT_BATCH_SEPARATE", None)
    ns = [F.fmmfft_plan_stats(h)["n"] for h in plans]
    out = {"metric": METRIC, "value": units / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c64 (fp32)", "data": "synthetic",
           "config": {"workload": BATCH_WL, "instances": len(plans),
                      "K_range": list(BATCH["K"]), "L_range": list(BATCH["L"]), "nrhs": BATCH["nrhs"],
                      "format": "tucker3d", "tol": BATCH["tol"],
                      "precision": "FP32 FFTs, 3xTF32 restores on the tensor cores",
                      "fft_extents": sorted({tuple(n) for n in ns}),
                      "fields_bytes": io_bytes, "setup_s": round(t_setup, 1),
                      "l2": "inputs and outputs larger than the 129 MB L2; no flush"},
           "per_step_ms": {"median": statistics.median(per), "min": min(per), "max": max(per)},
           "shared_launch_instances": shared,
           "separate_launches": {"ms_per_step": ms_sep, "value": units / (ms_sep * 1e-3) / 1e9},
           "clocks": clk}
    for h in plans:
        F.fmmfft_plan_destroy(h)
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nrhs", type=int, default=0, help="override the RHS count (profiling cases)")
    ap.add_argument("--L", type=int, default=-1, help="override the multipole count (profiling cases)")
    ap.add_argument("--only", default="both", choices=["both", "compressed", "plain"])
    ap.add_argument("--restore", default="", choices=["", "3xtf32", "bf16x3", "tf32", "fp32"],
                    help="restore arithmetic of the compressed arm (default: the workload's): tensor cores "
                         "(3xTF32, BF16x3, single TF32) or FP32 CUDA cores")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shard", default="directions", choices=["replicas", "directions"],
                    help="N > 1: the directions of one problem split into contiguous blocks, one shard plan "
                         "per GPU (default; strong scaling), or independent problems per GPU (weak scaling)")
    ap.add_argument("--no-farfield", action="store_true",
                    help="skip timing the aggregation / disaggregation steps (Eqs. 4, 6)")
    ap.add_argument("--no-occupancy", action="store_true",
                    help="skip timing the translation on a shell occupancy mask (Sec. II.A)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default schedule instead of autotuning each arm before timing")
    ap.add_argument("--workload", default=DEFAULT_WL, choices=sorted(WORKLOADS) + [BATCH_WL])
    ap.add_argument("--cpu-baseline-child", default="")
    ap.add_argument("--cpu-baseline-out", default="")
    ap.add_argument("--reference-child", nargs=3, default=None)
    args = ap.parse_args()
    if args.cpu_baseline_child:
        cpu_baseline_child(args.cpu_baseline_child, args.cpu_baseline_out)
        return
    if args.reference_child:
        reference_child(args.reference_child[0], int(args.reference_child[1]), int(args.reference_child[2]))
        return
    if args.impl == "reference":
        if args.workload == BATCH_WL:
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no oracle arm"}))
            return
        run_reference(args)
        return
    args.warmup = max(args.warmup, 3)
    if args.workload == BATCH_WL:
        run_batch(args)
        return

    import numpy as np
    import torch

    import paper_2010_00520_gb300 as F
    from seeded_inputs import field_spectra_torch

    from paper_2010_00520_gb300.replicas import (direction_block, job_throughput, max_over_ranks, ranks_from_env,
                                                 replica_seed)
    R_ = ranks_from_env()
    world, rank, local = R_.world, R_.rank, R_.local
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not os.path.exists(F.LIB_PATH):
        # one builder per node; the other ranks wait for it
        if local == 0:
            from paper_2010_00520_gb300 import build as _b
            _b.build()
        if dist is not None:
            dist.barrier()

    W = workload(args.workload)
    if args.L >= 0:
        W["L"] = args.L
        W["name"] = W["name"].replace(f"_L{WORKLOADS[args.workload]['L']}_", f"_L{args.L}_")
        args.no_cpu_baseline = True
    K, L, nrhs = W["K"], W["L"], (args.nrhs or W["nrhs"])
    shard = args.shard == "directions" and world > 1
    n_dir_grid = n_dir_of(W)
    first, count = direction_block(n_dir_grid, world, rank) if shard else (0, n_dir_grid)
    seed = W["seed"] if shard else replica_seed(W["seed"], rank)   # shards split one problem
    c128 = W.get("c128", False)
    fmt_c, dec_c = W["fmt"], W["dec"]
    restore = args.restore or W.get("restore", "3xtf32")
    plans = {}
    arms = [("plain", 0, 0, 0.0)]
    if fmt_c:
        arms.insert(0, ("compressed", fmt_c, dec_c, W["tol"]))
    arms = [a for a in arms if args.only in ("both", a[0])]
    t_setup = {}
    for name, fmt, dec, tol in arms:
        h = F.fmmfft_plan_create(K[0], K[1], K[2], W["a"], W["k0"], L, fmt, dec, tol)
        if c128:
            prec = F.FMMFFT_PREC_C128
        elif name == "compressed":
            prec = {"3xtf32": F.FMMFFT_PREC_C64_3XTF32, "bf16x3": F.FMMFFT_PREC_C64_BF16X3,
                    "tf32": F.FMMFFT_PREC_C64_TF32, "fp32": F.FMMFFT_PREC_C64}[restore]
        else:
            prec = F.FMMFFT_PREC_C64
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, prec)
        if shard:
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_DIR_FIRST, first)
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_DIR_COUNT, count)
        t0 = time.perf_counter()
        F.fmmfft_compress(h)
        t_setup[name] = time.perf_counter() - t0
        if not args.no_autotune:
            F.fmmfft_autotune(h, nrhs, 4000.0)
        plans[name] = h
    main_arm = "compressed" if "compressed" in plans else "plain"
    st = F.fmmfft_plan_stats(plans[main_arm])
    n, n_dir = tuple(st["n"]), st["n_dir"]
    sranks, pranks = (slab_ranks_of(F, plans["compressed"], fmt_c, dec_c, n_dir) if "compressed" in plans
                      else (None, None))
    tdt = torch.complex128 if c128 else torch.complex64
    stream = torch.cuda.current_stream()
    # seeded fields generated on the device (same values as the NumPy
    # generator the oracle uses); a shard's fields are its block of the problem's
    x = field_spectra_torch(seed, n_dir_grid, nrhs, K, first=first, count=count, device="cuda", dtype=tdt)
    y = torch.empty_like(x)
    io_bytes = x.numel() * x.element_size()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(h, steps):
        for _ in range(args.warmup):
            F.fmmfft_translate(h, x, y, nrhs, stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for i in range(steps):
            F.fmmfft_translate(h, x, y, nrhs, stream)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        ms = ev[0].elapsed_time(ev[steps]) / steps
        return max_over_ranks(ms, dist, "cuda"), per

    units = _units(n, n_dir, nrhs)

    # throughput of the job: shards count one problem, replicas every rank's,
    # in both cases timed by the slowest rank
    def job_value(seconds):
        if shard:
            return _units(n, n_dir_grid, nrhs) / seconds
        return job_throughput(units, world, seconds)

    def spread(v):
        q = statistics.quantiles(v, n=4) if len(v) >= 2 else [v[0]] * 3
        return {"median": statistics.median(v), "p25": q[0], "p75": q[2], "min": min(v), "max": max(v)}

    clocks = ClockSampler(local)
    clocks.start()
    ms, per_step = {}, {}
    for name, h in plans.items():
        ms[name], per_step[name] = timed(h, args.steps)
    clk = clocks.stop()
    for h in plans.values():
        assert F.fmmfft_poll_status(h) == 0
    value = {name: job_value(t * 1e-3) / 1e9 for name, t in ms.items()}


    # the same arm on the shell of boxes a meshed sphere occupies (Sec. II.A:
    # empty boxes carry no sources and receive nothing; x-lines with no
    # occupied box are pruned from both x passes)
    occupancy = None
    if not args.no_occupancy and world == 1:
        from seeded_inputs import shell_occupancy
        m = shell_occupancy(K)
        hm = plans[main_arm]
        F.fmmfft_plan_set_occupancy(hm, m)
        ms_m, per_m = timed(hm, args.steps)
        assert F.fmmfft_poll_status(hm) == 0
        F.fmmfft_plan_set_occupancy(hm, None)
        occupancy = {"mask": "shell of boxes within one box edge of the inscribed sphere",
                     "occupied_boxes": int(m.sum()), "boxes": int(m.size),
                     "occupied_x_lines": int(m.any(axis=2).sum()), "x_lines": int(K[1] * K[2]),
                     "ms_per_step": ms_m, "per_step_ms": spread(per_m),
                     "value": job_value(ms_m * 1e-3) / 1e9, "unit": UNIT,
                     "note": "same metric (padded voxels x fields / t): the pruned x-lines are not discounted"}

    # per-stage device times (CUDA events on the launch stream between the
    # kernels, which then run serially)
    stage = {}
    for name, h in plans.items():
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PROFILE, 1)
        acc = [0.0] * F.FMMFFT_NUM_STAGES
        nst = min(args.steps, 20)
        for _ in range(nst):
            F.fmmfft_translate(h, x, y, nrhs, stream)
            t = F.fmmfft_stage_times(h)
            acc = [a + b for a, b in zip(acc, t)]
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PROFILE, 0)
        stage[name] = {k: v / nst for k, v in zip(("restore", "xfwd", "yz", "xinv"), acc)}

    # far-field steps around the translation (Eqs. 4 and 6): synthetic patterns
    # of FAR_NB basis functions per box, the workload's spectra as B; only where
    # the patterns fit beside the fields
    farfield = None
    pat_bytes = n_dir * 2 * FAR_NB * K[0] * K[1] * K[2] * x.element_size()
    if not args.no_farfield and not c128 and world == 1 and pat_bytes <= 8e9:
        nb = FAR_NB
        g = torch.Generator(device="cuda").manual_seed(W["seed"])
        box = (K[2], K[1], K[0])
        Pd = torch.randn((n_dir, 2, nb) + box, dtype=tdt, device="cuda", generator=g)
        Id = torch.randn((nrhs, nb) + box, dtype=tdt, device="cuda", generator=g)
        Ad = torch.empty_like(x)
        Yd = torch.empty_like(Id)
        hf = plans[main_arm]

        def t_ff(fn):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            nf = min(args.steps, 50)
            e0.record(stream)
            for _ in range(nf):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / nf

        ms_agg = t_ff(lambda: F.fmmfft_aggregate(hf, Pd, Id, Ad, nb, nrhs, stream))
        ms_dis = t_ff(lambda: F.fmmfft_disaggregate(hf, Pd, x, Yd, nb, nrhs, stream))
        # Eq. 5 and Eq. 6 in one call: the translated fields stay on chip
        ms_tdis = t_ff(lambda: F.fmmfft_translate_disaggregate(hf, x, Pd, Yd, nb, nrhs, stream))
        pk = _peaks()[0].get("hbm_gbs", 6800.0)
        es = x.element_size()
        b_agg = (Pd.numel() + Id.numel() + Ad.numel()) * es
        b_dis = (Pd.numel() + x.numel() + Yd.numel()) * es
        farfield = {"nb": nb, "patterns_bytes": Pd.numel() * es,
                    "aggregate": {"ms": ms_agg, "algorithmic_bytes": b_agg,
                                  "achieved_gbs": b_agg / (ms_agg * 1e-3) / 1e9,
                                  "frac_of_hbm": b_agg / (ms_agg * 1e-3) / 1e9 / pk},
                    "disaggregate": {"ms": ms_dis, "algorithmic_bytes": b_dis,
                                     "achieved_gbs": b_dis / (ms_dis * 1e-3) / 1e9,
                                     "frac_of_hbm": b_dis / (ms_dis * 1e-3) / 1e9 / pk},
                    "far_field_matvec_ms": ms_agg + ms[main_arm] + ms_dis,
                    "translate_disaggregate_ms": ms_tdis,
                    "far_field_matvec_fused_ms": ms_agg + ms_tdis}
        del Pd, Id, Ad, Yd
        torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        # end to end through the host-buffer entry point: pinned host fields
        # in, the translated fields back in pinned host memory, every step
        hin = torch.empty(x.shape, dtype=tdt, pin_memory=True)
        hin.copy_(x)
        hout = torch.empty_like(hin, pin_memory=True)
        torch.cuda.synchronize()
        for _ in range(2):
            F.fmmfft_translate_host(plans[main_arm], hin, hout, nrhs, stream)
        barrier()
        ne = min(args.steps, 10)
        t0 = time.perf_counter()
        for _ in range(ne):
            F.fmmfft_translate_host(plans[main_arm], hin, hout, nrhs, stream)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / ne, dist, "cuda")
        e2e = {"value": job_value(e2e_s) / 1e9, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
               "d2h_bytes_per_step": io_bytes, "ms_per_step": e2e_s * 1e3,
               "entry_point": "fmmfft_translate_host (pinned host buffers, copies pipelined with the "
                              "translation over direction blocks)"}
        del hin, hout

    # ---- roofline --------------------------------------------------------
    peaks, peak_src = _peaks()
    props = torch.cuda.get_device_properties(local)
    sms = int(props.multi_processor_count)
    mhz = float(clk["sm_mhz"]) if clk.get("sm_mhz") else float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = fp32_peak_tflops(sms, mhz)
    yz_ms = stage[main_arm]["yz"]
    yz_fl = yz_fft_flops(K, n, n_dir, nrhs)
    achieved = yz_fl / (yz_ms * 1e-3) / 1e12
    large = bool(st.get("large_planes"))
    kname = "yzl_kernel" if large else "yz_kernel"
    traffic = None
    prof = os.path.join(ROOT, "profiles", f"{kname}_{W['name']}.traffic.json")
    if os.path.exists(prof) and main_arm == "compressed":
        with open(prof) as f:
            tj = json.load(f)
        # counters only count for the kernel and launch they were taken on
        if (tj.get("kernel_version") == YZ_KERNEL_VERSION[kname] and nrhs == W["nrhs"]
                and tj.get("restore_on_tensor_cores") == st.get("restore_on_tensor_cores")):
            traffic = tj.get("dram_bytes_per_launch")
    tc = int(st.get("restore_on_tensor_cores") or 0)
    tensor = None
    t_tc_ms = 0.0
    if main_arm == "compressed" and tc:
        split = 1 if tc == 3 else 3               # real MMAs per complex product
        slab_fl = 8 * slab_restore_macs(n, sranks) * split
        pre_fl = 8 * prepass_macs(n, n_dir, fmt_c, dec_c, pranks) * split
        tpk, tsrc = tensor_peak_tflops(peaks, "bf16x3" if tc == 2 else "tf32")
        t_tc_ms = (slab_fl + pre_fl) / (tpk * 1e12) * 1e3
        tensor = {"kernel": kname + " slab restores (tcgen05, " + {1: "3xTF32", 2: "BF16x3", 3: "TF32"}[tc] + ")",
                  "achieved": slab_fl / (yz_ms * 1e-3) / 1e12, "peak": tpk, "unit": "TFLOP/s",
                  "frac": slab_fl / (yz_ms * 1e-3) / 1e12 / tpk, "peak_source": tsrc,
                  "flops_model": f"8 flops per complex MAC x {split} real MMAs per product (split precision); "
                                 "averaged over the whole yz kernel time, which the FFTs share",
                  "prepass_flops_per_step": pre_fl}
    step_bytes = 2 * io_bytes + st["device_bytes_operator"]
    t_step = ms[main_arm]
    t_hbm = step_bytes / (peaks.get("hbm_gbs", 6800.0) * 1e9) * 1e3
    t_fp32 = step_fp32_flops(K, n, n_dir, nrhs) / (fp32_peak * 1e12) * 1e3
    bind = max((t_hbm, "hbm"), (t_fp32, "fp32"), (t_tc_ms, "tensor"))
    out = {
        "metric": METRIC, "value": value[main_arm], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms[main_arm], "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "c128 (fp64)" if c128 else "c64 (fp32)", "data": "synthetic",
        "config": dict(config_of(W, nrhs, world,
                                 (f"direction shards over {world} GPUs (rank 0: directions {first}..{first + count - 1})"
                                  if shard else (f"{world} replicas" if world > 1 else "1 GPU"))),
                       precision=("FP64 FFTs" if c128 else
                                  "FP32 FFTs, 3xTF32 restores on the tensor cores (tcgen05, FP32 accumulate)"
                                  if tc == 1 else
                                  "FP32 FFTs, BF16x3 restores on the tensor cores (tcgen05, FP32 accumulate)"
                                  if tc == 2 else
                                  "FP32 FFTs, single-TF32 restores on the tensor cores (ablation)"
                                  if tc == 3 else "FP32 FFTs and FP32 restores"),
                       large_planes=large,
                       schedule={name: dict(zip(("xrows", "tc_slab", "tc_gemm", "serial_prepass"),
                                                [int(v) for v in F.fmmfft_plan_stats(h)["schedule"]]))
                                 for name, h in plans.items()},
                       setup_s={k: round(v, 2) for k, v in t_setup.items()},
                       l2=("inputs and outputs each larger than the 129 MB L2; no flush" if io_bytes > 129e6 else
                           "inputs smaller than L2 (parity-sized workload); no flush")),
        "per_step_ms": {name: spread(v) for name, v in per_step.items()},
        "stages_ms": stage,
        "roofline": {"kernel": kname + " (y/z FFTs + Hadamard, FP32 CUDA cores)",
                     "bound": "alu",
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": traffic,
                     "peak_source": f"FP32 FMA peak {sms} SMs x 128 lanes x 2 flops x {mhz:.0f} MHz "
                                    f"(SM count from the device, median SM clock sampled during the timed region)",
                     "flops_model": "nominal 5 N log2 N per complex DFT line + 6 per Hadamard point, FP32 work "
                                    "only; the restores' tensor-core work is under roofline.tensor",
                     "tensor": tensor,
                     "step": {"t_hbm_ms": t_hbm, "t_fp32_ms": t_fp32, "t_tensor_ms": t_tc_ms, "t_step_ms": t_step,
                              "binding": bind[1], "frac": bind[0] / t_step,
                              "note": "max(t_HBM, t_FP32, t_TC) / t: HBM at the measured copy bandwidth over "
                                      "fields in + out + stored operator, FP32 over both x passes and the yz "
                                      "FFT + Hadamard flops, tensor over slab restore + pre-pass flops"}},
        "hbm": {"algorithmic_bytes_per_step": step_bytes,
                "achieved_gbs": step_bytes / (ms[main_arm] * 1e-3) / 1e9,
                "peak_gbs": peaks.get("hbm_gbs"), "peak_source": peak_src,
                "frac": step_bytes / (ms[main_arm] * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6800.0)},
        "clocks": clk,
        "gpu_launches": int(st["kernel_launches"]) * args.steps,
    }
    if "plain" in plans and "compressed" in plans:
        out["plain"] = {"value": value["plain"], "ms_per_step": ms["plain"]}
        out["ratio_compressed_over_plain_time"] = ms["compressed"] / ms["plain"]
        out["memory"] = {"operator_bytes_compressed": st["device_bytes_operator"],
                         "operator_bytes_plain": F.fmmfft_plan_stats(plans["plain"])["device_bytes_operator"],
                         "saving": st["saving"], "max_rank": [int(v) for v in st["max_rank"] if v],
                         "mean_rank": [round(v, 2) for v in st["mean_rank"]]}
    if e2e is not None:
        out["e2e"] = e2e
    if farfield is not None:
        out["farfield"] = farfield
    if occupancy is not None:
        out["occupancy_shell"] = occupancy
    if rank == 0 and world == 1 and not args.no_cpu_baseline and nrhs == W["nrhs"]:
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            ref_path = os.path.join(td, "oracle_fields.npz")
            out["cpu_baseline"] = run_cpu_baseline(W["name"], ref_path)
            if os.path.exists(ref_path):
                # accuracy of the timed outputs on the oracle's sample of
                # fields: the GPU translation against the uncompressed FP64 one
                ref = np.load(ref_path)
                dirs = [int(d) for d in ref["dirs"]]
                fsel = ref["fields"]
                exact = ref["exact"]
                acc = {"fields": int(exact.shape[0] * exact.shape[1]), "directions": dirs,
                       "oracle": ("its own Tucker-3D compression" if oracle_mode(W) == "tucker3d"
                                  else "uncompressed FP64 operator")}
                nf = 2 * nrhs
                for name, h in plans.items():
                    F.fmmfft_translate(h, x, y, nrhs, stream)
                    torch.cuda.synchronize()
                    got = np.stack([y[p].reshape((nf,) + tuple(y.shape[3:]))[torch.as_tensor(fsel[i])]
                                    .cpu().numpy().astype(np.complex128) for i, p in enumerate(dirs)])
                    acc[f"{name}_rel_l2_vs_fp64"] = float(np.linalg.norm(got - exact) / np.linalg.norm(exact))
                if oracle_mode(W) == "tucker3d":
                    acc["oracle_compressed_rel_l2_vs_fp64"] = float(np.linalg.norm(ref["oracle"] - exact)
                                                                    / np.linalg.norm(exact))
                out["accuracy"] = acc
    for h in plans.values():
        F.fmmfft_plan_destroy(h)
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
