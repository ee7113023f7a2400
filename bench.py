#!/usr/bin/env python
"""Throughput of the compressed FMM-FFT translation stage on GPUs of one node.

One step = one fmmfft_translate call: every field of the workload (all
directions, both polarisations, every RHS) translated through Eq. 5 with the
operator restored from its Tucker-3D compression (Sec. II.C).  The
uncompressed (plain) translation of the same workload is timed beside it.

Workload (default): 32^3 boxes of edge 0.5 wavelength (k0 = 2 pi), L = 8,
162 directions (Gauss-Legendre x 18 uniform phi), FFT grid 64^3, Tucker-3D
HOSVD at tol 1e-4, complex64 fields with FP32 FFTs and restores, 2
polarisations x 4 RHS of seeded i.i.d. complex Gaussian box spectra
(synthetic stand-ins for the aggregated fields of a meshed structure).

Metric: Gvoxel.dir/s = n1 n2 n3 * n_dir * 2 * nrhs / t / 1e9 (padded voxels
times fields translated per second).  Inputs (340 MB) and outputs (340 MB) are
each larger than the 129 MB L2, so no flush is needed between steps.

Launch: python bench.py [--gpus N --steps K --warmup W] (torchrun for N > 1:
every rank translates its own copy of the workload, weak scaling, no
collective on the data path).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
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
# workload has only the plain arm); c128: complex128 arithmetic.
WORKLOADS = {
    # the headline: Tucker-3D per direction, 3xTF32 restores
    "tucker3d_32cube_L8_tol1e-4_2pol_4rhs": dict(K=(32, 32, 32), L=8, tol=1e-4, nrhs=4, seed=1002, fmt=3, dec=1),
    "plain_c128_8cube_L5_2pol_1rhs": dict(K=(8, 8, 8), L=5, tol=0.0, nrhs=1, seed=1001, fmt=0, dec=0, c128=True),
    "tt4d_64cube_L10_tol1e-3_2pol_1rhs": dict(K=(64, 64, 64), L=10, tol=1e-3, nrhs=1, seed=1003, fmt=4, dec=2),
    "htucker4d_64cube_L10_tol1e-3_2pol_1rhs": dict(K=(64, 64, 64), L=10, tol=1e-3, nrhs=1, seed=1003, fmt=4, dec=3),
    "tucker3d_128x128x32_L6_tol1e-4_2pol_16rhs": dict(K=(128, 128, 32), L=6, tol=1e-4, nrhs=16, seed=1005,
                                                     fmt=3, dec=1),
    "htucker4d_128x128x32_L6_tol1e-4_2pol_16rhs": dict(K=(128, 128, 32), L=6, tol=1e-4, nrhs=16, seed=1005,
                                                      fmt=4, dec=3),
}
DEFAULT_WL = "tucker3d_32cube_L8_tol1e-4_2pol_4rhs"
WL = dict(WORKLOADS[DEFAULT_WL], name=DEFAULT_WL, a=0.5, k0=2 * math.pi)
FORMAT_NAMES = {(3, 1): "tucker3d", (3, 2): "tt3d", (4, 1): "tucker4d", (4, 2): "tt4d", (4, 3): "htucker4d",
                (0, 0): "none"}
FAR_NB = 16                  # basis functions per box of the far-field steps (Eqs. 4, 6)
CPU_SAMPLE_DIRS = 8          # directions (x 8 fields) the CPU baseline translates
# version of the yz kernel the committed DRAM-traffic figure was taken on
YZ_KERNEL_VERSION = 5


def _units(n, n_dir, nrhs):
    return n[0] * n[1] * n[2] * n_dir * 2 * nrhs


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
# CPU baseline: the FP64 oracle, one thread, on a bounded sample
# ---------------------------------------------------------------------------
def cpu_baseline_child(ndirs: int, out_path: str = ""):
    """Runs in a subprocess with one BLAS/OpenMP thread.  Times the oracle's
    compressed translation (Tucker-3D restore of each sampled direction, Fig.
    3(a), then Eq. 5 for its 8 fields); the oracle's HOSVD set-up is not
    timed, as the GPU arm's set-up is not.  Afterwards (untimed) it translates
    the same fields with the uncompressed FP64 operators and, given out_path,
    saves both results there (.npz) so that the GPU outputs of these fields
    can be checked against them."""
    import numpy as np
    from oracle import decomp as D
    from oracle import pipeline as pl
    from oracle import translate as tr
    from seeded_inputs import field_spectra_rows

    K, L, nrhs, seed = WL["K"], WL["L"], WL["nrhs"], WL["seed"]
    plan = pl.Plan(K=K, L=L)
    dirs = [int(round(i * (plan.n_dir - 1) / max(ndirs - 1, 1))) for i in range(ndirs)]
    ops = pl.operators(plan, dirs)
    tks = [D.tucker_hosvd(T, WL["tol"]) for T in ops]
    nf = 2 * nrhs
    fields = np.array([p * nf + j for p in dirs for j in range(nf)])
    A = field_spectra_rows(seed, plan.n_dir, nrhs, K, fields)
    comp = []
    t0 = time.perf_counter()
    i = 0
    for tk in tks:
        That = D.tucker3d_restore_steps(tk.core, *tk.factors)
        for _ in range(nf):
            comp.append(tr.translate_field_fft(That, A[i]))
            i += 1
    dt = time.perf_counter() - t0
    n = plan.n
    units = n[0] * n[1] * n[2] * len(fields)
    if out_path:
        exact = [tr.translate_field_fft(ops[k], A[k * nf + j]) for k in range(len(dirs)) for j in range(nf)]
        np.savez(out_path, dirs=np.array(dirs), compressed=np.stack(comp), exact=np.stack(exact))
    print(json.dumps({"seconds": dt, "units": units, "fields": int(len(fields)), "dirs": len(dirs)}))


def run_cpu_baseline(ndirs: int, out_path: str = ""):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-child", str(ndirs)]
    if out_path:
        cmd += ["--cpu-baseline-out", out_path]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["units"] / d["seconds"] / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "seconds": d["seconds"],
            "sample": f"{d['dirs']} of 162 directions x 8 fields (2 pol x 4 RHS) of the 32^3-box L=8 "
                      f"workload: Tucker-3D restore + FFT translation, FP64 NumPy, 1 thread"}


# ---------------------------------------------------------------------------
# reference arm: the oracle as the reference implementation
# ---------------------------------------------------------------------------
def reference_child(steps: int, warmup: int):
    """One BLAS thread.  A step translates one field of the workload with the
    oracle (Eq. 5, FP64), its direction's Tucker-3D operator restored (Fig.
    3(a)) whenever the direction changes; fields are taken in workload order
    starting at direction 0.  Prints the per-step seconds."""
    import numpy as np
    from oracle import decomp as D
    from oracle import pipeline as pl
    from oracle import translate as tr
    from seeded_inputs import field_spectra_rows

    K, L, nrhs, seed = WL["K"], WL["L"], WL["nrhs"], WL["seed"]
    plan = pl.Plan(K=K, L=L)
    nf = 2 * nrhs
    total = steps + warmup
    dirs = sorted({f // nf for f in range(total)})
    tks = {p: D.tucker_hosvd(pl.operators(plan, [p])[0], WL["tol"]) for p in dirs}
    A = field_spectra_rows(seed, plan.n_dir, nrhs, K, np.arange(total))
    secs = []
    cur, That = None, None
    for f in range(total):
        t0 = time.perf_counter()
        p = f // nf
        if p != cur:
            tk = tks[p]
            That = D.tucker3d_restore_steps(tk.core, *tk.factors)
            cur = p
        tr.translate_field_fft(That, A[f])
        secs.append(time.perf_counter() - t0)
    print(json.dumps({"seconds": secs[warmup:]}))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--reference-child",
                        str(args.steps), str(args.warmup)],
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + r.stderr[-300:]}))
        return
    secs = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
    units = 64 ** 3
    val = units * len(secs) / sum(secs) / 1e9
    sample = (f"{len(secs)} fields (one per step) of the 32^3-box L=8 Tucker-3D workload, taken in "
              f"workload order; FP64 NumPy oracle (restore + FFT translation), 1 thread")
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": WL["name"], "K": list(WL["K"]), "L": WL["L"], "n_dir": 162,
                      "nrhs": WL["nrhs"], "tol": WL["tol"], "step": "one field of the workload per step"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# flop / byte models of one step (nominal 5 N log2 N flops per complex DFT)
# ---------------------------------------------------------------------------
def yz_flops(K, n, n_dir, nrhs, slab_ranks=None):
    """Nominal flops of one yz launch.  slab_ranks: per direction (ra, rb) of
    the slab restore (Tucker-like: ra = r2, rb = r3; TT-like: ra = 0, rb = r2)."""
    Kx, Ky, Kz = K
    n1, n2, n3 = n
    lg2, lg3 = math.log2(n2), math.log2(n3)
    per_field_slab = 2 * Kz * 5 * n2 * lg2 + n2 * (2 * 5 * n3 * lg3 + 6 * n3)
    f = n1 * n_dir * 2 * nrhs * per_field_slab
    if slab_ranks is not None:
        # per block: (n2 x ra)(ra x rb) when ra > 0, then (n3 x rb)(rb x n2); 8 flops per complex MAC
        f += n1 * sum(8 * (n2 * ra * rb + n3 * n2 * rb) for (ra, rb) in slab_ranks)
    return f


def step_flops(K, n, n_dir, nrhs, slab_ranks=None):
    Kx, Ky, Kz = K
    n1, n2, n3 = n
    F = n_dir * 2 * nrhs
    x = F * 2 * Ky * Kz * 5 * n1 * math.log2(n1)
    return x + yz_flops(K, n, n_dir, nrhs, slab_ranks)


def slab_ranks_of(F, h, fmt, dec, n_dir):
    st = F.fmmfft_plan_stats(h)
    r = st["max_rank"]
    if fmt == 3:
        pr = F.fmmfft_plan_ranks(h)
        return [(int(a[1]), int(a[2])) if dec == 1 else (0, int(a[1])) for a in pr]
    if dec == 2:
        return [(0, int(r[1]))] * n_dir
    return [(int(r[1]), int(r[2]))] * n_dir


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nrhs", type=int, default=0, help="override the RHS count (profiling cases)")
    ap.add_argument("--only", default="both", choices=["both", "compressed", "plain"])
    ap.add_argument("--restore", default="3xtf32", choices=["3xtf32", "bf16x3", "tf32", "fp32"],
                    help="restore arithmetic of the compressed arm: tensor cores (3xTF32 or BF16x3) or FP32 CUDA cores")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "directions"],
                    help="N > 1: independent problems per GPU (weak scaling) or the directions of one "
                         "problem split into contiguous blocks, one shard plan per GPU (strong scaling)")
    ap.add_argument("--no-farfield", action="store_true",
                    help="skip timing the aggregation / disaggregation steps (Eqs. 4, 6)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default schedule instead of autotuning each arm before timing")
    ap.add_argument("--workload", default=DEFAULT_WL, choices=sorted(WORKLOADS),
                    help="workload (default: the headline Tucker-3D one); others print their own line "
                         "without CPU baseline and end-to-end arms")
    ap.add_argument("--cpu-baseline-child", type=int, default=0)
    ap.add_argument("--cpu-baseline-out", default="")
    ap.add_argument("--reference-child", type=int, nargs=2, default=None)
    args = ap.parse_args()
    if args.cpu_baseline_child:
        cpu_baseline_child(args.cpu_baseline_child, args.cpu_baseline_out)
        return
    if args.reference_child:
        reference_child(*args.reference_child)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch

    import paper_2010_00520_gb300 as F
    from seeded_inputs import field_spectra

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

    wl_name = args.workload
    W = dict(WORKLOADS[wl_name], a=0.5, k0=2 * math.pi)
    if wl_name != DEFAULT_WL:
        args.no_e2e = True
        args.no_cpu_baseline = True
        args.no_farfield = True
    K, L, nrhs = W["K"], W["L"], (args.nrhs or W["nrhs"])
    shard = args.shard == "directions" and world > 1
    n_dir_grid = 2 * (L + 1) ** 2
    first, count = direction_block(n_dir_grid, world, rank) if shard else (0, n_dir_grid)
    seed = W["seed"] if shard else replica_seed(W["seed"], rank)   # shards split one problem
    c128 = W.get("c128", False)
    fmt_c, dec_c = W["fmt"], W["dec"]
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
        elif name == "compressed" and args.restore == "3xtf32":
            prec = F.FMMFFT_PREC_C64_3XTF32
        elif name == "compressed" and args.restore == "bf16x3":
            prec = F.FMMFFT_PREC_C64_BF16X3
        elif name == "compressed" and args.restore == "tf32":
            prec = F.FMMFFT_PREC_C64_TF32
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
            F.fmmfft_autotune(h, args.nrhs or W["nrhs"], 4000.0)
        plans[name] = h
    main_arm = "compressed" if "compressed" in plans else "plain"
    st = F.fmmfft_plan_stats(plans[main_arm])
    n, n_dir = tuple(st["n"]), st["n_dir"]
    sranks = slab_ranks_of(F, plans["compressed"], fmt_c, dec_c, n_dir) if "compressed" in plans else None
    cdt = np.complex128 if c128 else np.complex64
    tdt = torch.complex128 if c128 else torch.complex64
    stream = torch.cuda.current_stream()
    S_host = None
    if wl_name == DEFAULT_WL:
        # a shard's fields are its block of the whole problem's
        S_host = field_spectra(seed, n_dir_grid, nrhs, K)[first:first + count].astype(cdt)
        x = torch.from_numpy(np.ascontiguousarray(S_host)).to("cuda")
    else:
        # generated one direction at a time straight into device memory
        from seeded_inputs import field_spectra_rows
        x = torch.empty((n_dir, 2, nrhs, K[2], K[1], K[0]), dtype=tdt, device="cuda")
        nf = 2 * nrhs
        for p in range(n_dir):
            q = first + p
            rows = field_spectra_rows(seed, n_dir_grid, nrhs, K, np.arange(q * nf, (q + 1) * nf))
            x[p] = torch.from_numpy(rows.astype(cdt).reshape(2, nrhs, K[2], K[1], K[0])).to("cuda")
    y = torch.empty_like(x)
    io_bytes = x.numel() * x.element_size()

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(h, steps):
        for _ in range(args.warmup):
            F.fmmfft_translate(h, x, y, nrhs, stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            F.fmmfft_translate(h, x, y, nrhs, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / steps
        return max_over_ranks(ms, dist, "cuda")

    units = _units(n, n_dir, nrhs)
    # throughput of the job: replicas count every rank's problem, shards one
    # problem, in both cases timed by the slowest rank
    def job_value(seconds):
        if shard:
            return _units(n, n_dir_grid, nrhs) / seconds
        return job_throughput(units, world, seconds)
    clocks = ClockSampler(local)
    clocks.start()
    ms = {name: timed(h, args.steps) for name, h in plans.items()}
    clk = clocks.stop()
    for h in plans.values():
        assert F.fmmfft_poll_status(h) == 0
    value = {name: job_value(t * 1e-3) / 1e9 for name, t in ms.items()}

    # per-stage device times (CUDA events on the launch stream, between kernels)
    stage = {}
    for name, h in plans.items():
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PROFILE, 1)
        acc = [0.0] * F.FMMFFT_NUM_STAGES
        nst = min(args.steps, 50)
        for _ in range(nst):
            F.fmmfft_translate(h, x, y, nrhs, stream)
            t = F.fmmfft_stage_times(h)
            acc = [a + b for a, b in zip(acc, t)]
        F.fmmfft_plan_set(h, F.FMMFFT_KEY_PROFILE, 0)
        stage[name] = {k: v / nst for k, v in zip(("restore", "xfwd", "yz", "xinv"), acc)}

    # far-field steps around the translation (Eqs. 4 and 6): synthetic patterns
    # of FAR_NB basis functions per box, the workload's spectra as B
    farfield = None
    if not args.no_farfield and not c128 and world == 1:
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
                    "far_field_matvec_ms": ms_agg + ms[main_arm] + ms_dis}
        del Pd, Id, Ad, Yd

    e2e = None
    if not args.no_e2e:
        # end to end through the host-buffer entry point (pinned memory)
        hin = torch.from_numpy(S_host).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        for _ in range(2):
            F.fmmfft_translate_host(plans[main_arm], hin, hout, nrhs, stream)
        barrier()
        ne = min(args.steps, 50)
        t0 = time.perf_counter()
        for _ in range(ne):
            F.fmmfft_translate_host(plans[main_arm], hin, hout, nrhs, stream)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / ne, dist, "cuda")
        e2e = {"value": job_value(e2e_s) / 1e9, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
               "d2h_bytes_per_step": io_bytes}

    peaks, peak_src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12        # TFLOP/s, FMA = 2 flops
    yz_ms = stage[main_arm]["yz"]
    yz_fl = yz_flops(K, n, n_dir, nrhs, sranks)
    achieved = yz_fl / (yz_ms * 1e-3) / 1e12
    traffic = None
    prof = os.path.join(ROOT, "profiles", "yz_kernel_tucker3d_32cube_L8.traffic.json")
    if os.path.exists(prof) and main_arm == "compressed":
        with open(prof) as f:
            tj = json.load(f)
        # counters only count for the kernel they were taken on
        if (tj.get("kernel_version") == YZ_KERNEL_VERSION and wl_name == DEFAULT_WL and nrhs == W["nrhs"]
                and st.get("restore_on_tensor_cores") == 1):
            traffic = tj.get("dram_bytes_per_launch")
    step_bytes = 2 * io_bytes + st["device_bytes_operator"]
    out = {
        "metric": METRIC, "value": value[main_arm], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms[main_arm], "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "c128 (fp64)" if c128 else "c64 (fp32)", "data": "synthetic",
        "config": {"workload": wl_name if nrhs == W["nrhs"] else wl_name.replace(f"{W['nrhs']}rhs", f"{nrhs}rhs"),
                   "K": list(K), "n": list(n), "L": L, "n_dir": n_dir_grid,
                   "parallelism": (f"direction shards over {world} GPUs (rank 0: directions {first}..{first + count - 1})"
                                   if shard else (f"{world} replicas" if world > 1 else "1 GPU")),
                   "nrhs": nrhs, "fields": n_dir * 2 * nrhs,
                   "format": FORMAT_NAMES[(fmt_c, dec_c)] if main_arm == "compressed" else "none",
                   "tol": W["tol"],
                   "precision": ("FP64 FFTs" if c128 else
                                 "FP32 FFTs, 3xTF32 restores on the tensor cores (tcgen05, FP32 accumulate)"
                                 if st.get("restore_on_tensor_cores") == 1 else
                                 "FP32 FFTs, BF16x3 restores on the tensor cores (tcgen05, FP32 accumulate)"
                                 if st.get("restore_on_tensor_cores") == 2 else
                                 "FP32 FFTs, single-TF32 restores on the tensor cores (ablation)"
                                 if st.get("restore_on_tensor_cores") == 3 else "FP32 FFTs and FP32 restores"),
                   "large_planes": bool(st.get("large_planes")),
                   "schedule": {name: dict(zip(("xrows", "tc_slab", "tc_gemm", "serial_prepass"),
                                               [int(v) for v in F.fmmfft_plan_stats(h)["schedule"]]))
                                for name, h in plans.items()},
                   "setup_s": {k: round(v, 2) for k, v in t_setup.items()},
                   "l2": ("inputs and outputs each larger than the 129 MB L2; no flush" if io_bytes > 129e6 else
                          "inputs smaller than L2 (parity-sized workload); no flush")},
        "stages_ms": stage,
        "roofline": {"kernel": "yz_kernel (slab restore + y/z FFTs + Hadamard)",
                     "bound": "alu",
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": traffic,
                     "peak_source": f"FP32 FMA peak 152 SMs x 128 lanes x 2 x {sm_max:.0f} MHz ({peak_src} clock)",
                     "flops_model": "nominal 5 N log2 N per complex DFT line + 6 per Hadamard point + 8 per complex MAC of the restore"},
        "hbm": {"algorithmic_bytes_per_step": step_bytes,
                "achieved_gbs": step_bytes / (ms[main_arm] * 1e-3) / 1e9,
                "peak_gbs": peaks.get("hbm_gbs"),
                "frac": step_bytes / (ms[main_arm] * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6800.0)},
        "step_tflops_nominal": step_flops(K, n, n_dir, nrhs, sranks) / (ms[main_arm] * 1e-3) / 1e12,
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
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            ref_path = os.path.join(td, "oracle_fields.npz")
            out["cpu_baseline"] = run_cpu_baseline(CPU_SAMPLE_DIRS, ref_path)
            if os.path.exists(ref_path) and wl_name == DEFAULT_WL and nrhs == W["nrhs"]:
                # accuracy of the timed outputs on the oracle's sample of fields:
                # the GPU translation against the uncompressed FP64 one
                ref = np.load(ref_path)
                dirs = [int(d) for d in ref["dirs"]]
                acc = {"fields": int(ref["exact"].shape[0]), "directions": dirs}
                exact = ref["exact"]
                for name, h in plans.items():
                    F.fmmfft_translate(h, x, y, nrhs, stream)
                    torch.cuda.synchronize()
                    got = y[dirs].cpu().numpy().astype(np.complex128).reshape(exact.shape)
                    acc[f"{name}_rel_l2_vs_fp64"] = float(np.linalg.norm(got - exact) / np.linalg.norm(exact))
                acc["oracle_compressed_rel_l2_vs_fp64"] = float(np.linalg.norm(ref["compressed"] - exact)
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
