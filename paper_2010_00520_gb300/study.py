"""Compression study of the FFT'ed translation operators (Sec. III.A).

Ranks, memory saving and restore cost of the five compressed formats while one
parameter of the operator set varies, as in the paper's sphere study:

  * structure size (Table II, Figs. 5(a)-(d)): sphere diameter D, boxes per
    axis K = D / a, tensors n = 2K per axis;
  * decomposition tolerance gamma (Fig. 6);
  * FMM box size a (Fig. 7) at a fixed diameter;
  * FMM accuracy in digits (Fig. 8), which sets L and N_dir;
  * loss of the medium, relative permittivity 2 ... 2 - 8j (Table IV, Fig. 9).

Defaults are the paper's settings (Sec. III): 0.5-lambda boxes, 5 digits,
gamma = 1e-6, N_dir = (L+1)(2L+1) directions, L from the excess-bandwidth rule
of Sec. II.A, and the near-field rule R < kappa R^s with kappa = 4.

Host side, no GPU: the library's FP64 set-up (fmmfft_compress_host) gives the
ranks and the memory saving 1 - compressed / original.  With a GPU, every case
is also translated with its compressed and its plain operator on the same
synthetic fields and timed with CUDA events.  The paper's computational
overhead is the decompression time over the convolution time of a CPU code that
restores each direction before convolving with it; here the restore runs fused
inside the convolution kernels, so the overhead reported is
t_compressed / t_plain - 1 (negative where streaming the plain operator from
memory costs more than restoring it on chip).

Extents are powers of two (the embedding rule of the library), so box sizes
whose K = D / a is not a power of two are rounded up to the next one for n.

    python -m paper_2010_00520_gb300.study size --diameters 8 16 --formats all
    python -m paper_2010_00520_gb300.study loss --diameter 8 --gpu
"""
from __future__ import annotations

import argparse
import json
import math
from dataclasses import asdict, dataclass, field

import numpy as np

from . import (FMMFFT_FORMAT_3D, FMMFFT_FORMAT_4D, FMMFFT_FORMAT_NONE, FMMFFT_DECOMP_HTUCKER,
               FMMFFT_DECOMP_NONE, FMMFFT_DECOMP_TT, FMMFFT_DECOMP_TUCKER, FMMFFT_KEY_EPS_R_IM,
               FMMFFT_KEY_EPS_R_RE, FMMFFT_KEY_KAPPA, FMMFFT_KEY_NEAR_RULE, FMMFFT_KEY_NPHI_RULE,
               FMMFFT_KEY_PRECISION, FMMFFT_KEY_RESTORE_ERROR, FMMFFT_KEY_TRUNC_RULE, FMMFFT_PREC_C64,
               FMMFFT_PREC_C128,
               FMMFFT_ERR_UNSUPPORTED,
               FmmfftError, fmmfft_compress,
               fmmfft_compress_host, fmmfft_multipole_count, fmmfft_plan_create, fmmfft_plan_destroy,
               fmmfft_plan_set, fmmfft_plan_stats, fmmfft_translate)

WAVELENGTH = 1.0
K0 = 2 * math.pi / WAVELENGTH

# the five methodologies of Sec. II.B, in the paper's order
FORMATS = {
    "tt3d": (FMMFFT_FORMAT_3D, FMMFFT_DECOMP_TT),
    "tucker3d": (FMMFFT_FORMAT_3D, FMMFFT_DECOMP_TUCKER),
    "tt4d": (FMMFFT_FORMAT_4D, FMMFFT_DECOMP_TT),
    "tucker4d": (FMMFFT_FORMAT_4D, FMMFFT_DECOMP_TUCKER),
    "htucker": (FMMFFT_FORMAT_4D, FMMFFT_DECOMP_HTUCKER),
}


@dataclass
class StudyCase:
    """One operator set and one methodology."""
    fmt: str                      # key of FORMATS
    K: int                        # boxes per axis (cubic grid)
    a: float = 0.5                # box edge in wavelengths
    digits: float = 5.0           # FMM accuracy
    eps_r: complex = 1.0          # relative permittivity of the medium
    tol: float = 1e-6             # decomposition tolerance gamma
    nphi_rule: int = 1            # 1: N_dir = (L+1)(2L+1) (Sec. II.A)
    near_rule: int = 1            # 1: near iff R < kappa R^s
    kappa: float = 4.0
    trunc_rule: int = 0           # 0: discarded energy, 1: singular value
    L: int | None = None          # None: excess-bandwidth rule

    def multipoles(self) -> int:
        if self.L is not None:
            return self.L
        return fmmfft_multipole_count(self.a * WAVELENGTH, K0, self.digits, self.eps_r)


@dataclass
class StudyRow:
    case: dict
    L: int
    n: list
    n_dir: int
    ranks: list                   # 3D: largest (r1, r2, r3) over directions; 4D: the ranks
    mean_ranks: list
    elements_plain: int
    elements_compressed: int
    saving: float
    setup_s: float
    gpu: dict = field(default_factory=dict)
    restore_rel_err: float = -1.0  # FP64 error of the stored operator (-1: not measured)


def _configure(h, c: StudyCase, precision=None):
    e = complex(c.eps_r)
    opts = [(FMMFFT_KEY_NPHI_RULE, c.nphi_rule), (FMMFFT_KEY_NEAR_RULE, c.near_rule),
            (FMMFFT_KEY_KAPPA, c.kappa), (FMMFFT_KEY_TRUNC_RULE, c.trunc_rule),
            (FMMFFT_KEY_EPS_R_RE, e.real), (FMMFFT_KEY_EPS_R_IM, e.imag)]
    if precision is not None:
        opts.append((FMMFFT_KEY_PRECISION, precision))
    for k, v in opts:
        fmmfft_plan_set(h, k, v)


def _plan(c: StudyCase, L: int, fmt_dec, tol, precision=None):
    h = fmmfft_plan_create(c.K, c.K, c.K, c.a * WAVELENGTH, K0, L, fmt_dec[0], fmt_dec[1], tol)
    try:
        _configure(h, c, precision)
    except Exception:
        fmmfft_plan_destroy(h)
        raise
    return h


def host_case(c: StudyCase, restore_error: bool = False) -> StudyRow:
    """Ranks and memory saving of one case from the library's FP64 set-up;
    with restore_error also the FP64 relative error of the stored operator
    against the uncompressed one (the quantity the tolerance bounds), which
    costs one host restoration of every direction."""
    L = c.multipoles()
    h = _plan(c, L, FORMATS[c.fmt], c.tol)
    try:
        if restore_error:
            fmmfft_plan_set(h, FMMFFT_KEY_RESTORE_ERROR, 1)
        r, _ = fmmfft_compress_host(h, restored=False)
        st = fmmfft_plan_stats(h)
        setup = float(st["setup_seconds"])      # the set-up alone, without the error measurement
        if FORMATS[c.fmt][0] == FMMFFT_FORMAT_3D:
            ranks = [int(v) for v in r.max(axis=0)[: 3 if c.fmt == "tucker3d" else 2]]
            mean = [float(v) for v in r.mean(axis=0)[: len(ranks)]]
        else:
            used = {"tucker4d": 4, "htucker": 6, "tt4d": 3}[c.fmt]
            ranks = [int(v) for v in r[:used]]
            mean = []
        case = asdict(c)
        case["eps_r"] = [complex(c.eps_r).real, complex(c.eps_r).imag]
        return StudyRow(case=case, L=L, n=list(st["n"]), n_dir=st["n_dir"], ranks=ranks, mean_ranks=mean,
                        elements_plain=int(st["elements_plain"]), elements_compressed=int(st["elements_compressed"]),
                        saving=float(st["saving"]), setup_s=setup,
                        restore_rel_err=float(st["restore_rel_err"]))
    finally:
        fmmfft_plan_destroy(h)


def _time_translate(torch, h, x, y, nrhs, steps, warmup):
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        fmmfft_translate(h, x, y, nrhs, s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(steps):
        fmmfft_translate(h, x, y, nrhs, s)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def gpu_case(c: StudyCase, row: StudyRow, nrhs=1, precision=FMMFFT_PREC_C64, steps=20, warmup=3, seed=1234):
    """Time the compressed and the plain translation of one case on cuda:0 and
    add them to row.gpu (ms per translation of 2 polarisations x nrhs fields
    per direction; the inputs are seeded complex Gaussian fields in HBM)."""
    import torch

    L = row.L
    nd = row.n_dir
    g = torch.Generator(device="cuda").manual_seed(seed)
    shape = (nd, 2, nrhs, c.K, c.K, c.K)
    # fields in the plans' precision: complex128 for FMMFFT_PREC_C128
    cdt = torch.complex128 if precision == FMMFFT_PREC_C128 else torch.complex64
    x = torch.complex(torch.randn(shape, generator=g, device="cuda"),
                      torch.randn(shape, generator=g, device="cuda")).to(cdt)
    y = torch.empty_like(x)
    times = {}
    for name, fd, tol in (("compressed", FORMATS[c.fmt], c.tol),
                          ("plain", (FMMFFT_FORMAT_NONE, FMMFFT_DECOMP_NONE), 0.0)):
        h = _plan(c, L, fd, tol, precision)
        try:
            try:
                fmmfft_compress(h)
            except FmmfftError as e:
                if e.status != FMMFFT_ERR_UNSUPPORTED:
                    raise
                row.gpu = {"unsupported": str(e)}
                return row
            times[name] = _time_translate(torch, h, x, y, nrhs, steps, warmup)
        finally:
            fmmfft_plan_destroy(h)
    row.gpu = {"ms_compressed": times["compressed"], "ms_plain": times["plain"],
               "overhead": times["compressed"] / times["plain"] - 1.0, "nrhs": nrhs,
               "precision": precision}
    return row


# ---- the sweeps of Sec. III.A ------------------------------------------------

def _boxes(diameter, a):
    return int(round(diameter / a))


def structure_size(formats, diameters=(8, 16), **kw):
    """Table II / Fig. 5: sphere diameter in wavelengths, 0.5-lambda boxes."""
    return [StudyCase(fmt=f, K=_boxes(d, kw.get("a", 0.5)), **kw) for d in diameters for f in formats]


def tolerance(formats, gammas=(1e-3, 1e-4, 1e-5, 1e-6), diameter=8, **kw):
    """Fig. 6: decomposition tolerance."""
    kw.pop("tol", None)
    return [StudyCase(fmt=f, K=_boxes(diameter, kw.get("a", 0.5)), tol=g, **kw) for g in gammas for f in formats]


def box_size(formats, sizes=(0.25, 0.5, 1.0), diameter=8, **kw):
    """Fig. 7: FMM box edge in wavelengths at a fixed diameter."""
    kw.pop("a", None)
    return [StudyCase(fmt=f, K=_boxes(diameter, s), a=s, **kw) for s in sizes for f in formats]


def accuracy(formats, digits=(3, 4, 5, 6), diameter=8, **kw):
    """Fig. 8: FMM accuracy (digits), which sets L and the direction count."""
    kw.pop("digits", None)
    return [StudyCase(fmt=f, K=_boxes(diameter, kw.get("a", 0.5)), digits=dg, **kw) for dg in digits for f in formats]


def loss(formats, eps=(2.0, 2 - 1j, 2 - 2j, 2 - 8j), diameter=8, **kw):
    """Table IV / Fig. 9: relative permittivity of a lossy medium."""
    kw.pop("eps_r", None)
    return [StudyCase(fmt=f, K=_boxes(diameter, kw.get("a", 0.5)), eps_r=e, **kw) for e in eps for f in formats]


SWEEPS = {"size": structure_size, "tol": tolerance, "box": box_size, "digits": accuracy, "loss": loss}


def run(cases, gpu=False, nrhs=1, log=None, precision=FMMFFT_PREC_C64, restore_error=False):
    rows = []
    for c in cases:
        row = host_case(c, restore_error)
        if gpu:
            gpu_case(c, row, nrhs=nrhs, precision=precision)
        rows.append(row)
        if log:
            log(row)
    return rows


def table(rows) -> str:
    """Markdown table of study rows."""
    head = "| format | K | a | digits | eps_r | tol | L | N_dir | n | ranks | saving % | host set-up s |"
    gpu = any(r.gpu for r in rows)
    err = any(r.restore_rel_err >= 0 for r in rows)
    if err:
        head += " FP64 restore error |"
    if gpu:
        head += " ms compressed | ms plain | overhead |"
    out = [head, "|" + "---|" * (head.count("|") - 1)]
    for r in rows:
        c = r.case
        e = complex(*c["eps_r"])
        line = (f"| {c['fmt']} | {c['K']} | {c['a']:g} | {c['digits']:g} | {e.real:g}{e.imag:+g}j | {c['tol']:g} | "
                f"{r.L} | {r.n_dir} | {r.n[0]} | {tuple(r.ranks)} | {100 * r.saving:.2f} | {r.setup_s:.1f} |")
        if err:
            line += f" {r.restore_rel_err:.2e} |" if r.restore_rel_err >= 0 else " - |"
        if gpu:
            g = r.gpu
            if "ms_compressed" in g:
                line += f" {g['ms_compressed']:.3f} | {g['ms_plain']:.3f} | {g['overhead']:+.2f} |"
            else:
                line += " - | - | - |"
        out.append(line)
    return "\n".join(out)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("sweep", choices=sorted(SWEEPS))
    ap.add_argument("--formats", nargs="+", default=["tucker3d", "tt3d"],
                    help="methodologies (%s) or 'all'" % ", ".join(FORMATS))
    ap.add_argument("--diameters", nargs="+", type=float, default=[8, 16])
    ap.add_argument("--diameter", type=float, default=8)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--kappa", type=float, default=4.0)
    ap.add_argument("--near-rule", type=int, default=1)
    ap.add_argument("--trunc-rule", type=int, default=0)
    ap.add_argument("--gpu", action="store_true", help="also time compressed and plain translations")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--precision", type=int, default=FMMFFT_PREC_C64,
                    help="FMMFFT_PREC_*: 0 complex128, 1 complex64 with FP32 restores (default), 2 3xTF32, "
                         "3 BF16x3")
    ap.add_argument("--restore-error", action="store_true",
                    help="also measure the FP64 restore error of each stored operator (host)")
    ap.add_argument("--json", help="write the rows to this file")
    a = ap.parse_args(argv)
    fmts = list(FORMATS) if a.formats == ["all"] else a.formats
    kw = dict(kappa=a.kappa, near_rule=a.near_rule, trunc_rule=a.trunc_rule)
    if a.sweep == "size":
        cases = structure_size(fmts, a.diameters, tol=a.tol, **kw)
    elif a.sweep == "tol":
        cases = tolerance(fmts, diameter=a.diameter, **kw)
    else:
        cases = SWEEPS[a.sweep](fmts, diameter=a.diameter, tol=a.tol, **kw)
    rows = run(cases, gpu=a.gpu, nrhs=a.nrhs, precision=a.precision, restore_error=a.restore_error,
               log=lambda r: print(json.dumps(asdict(r)), flush=True))
    print(table(rows))
    if a.json:
        with open(a.json, "w") as f:
            json.dump([asdict(r) for r in rows], f, indent=1)


if __name__ == "__main__":
    main()
