"""Python binding of the compressed FMM-FFT translation library (libfmmfft.so).

The functions below carry the names of the C entry points declared in
include/fmmfft.h and only marshal arguments: every step of the translation
runs in the library's CUDA kernels.  Device buffers may be given as torch
tensors (their data_ptr() is used) or as integer addresses; streams as torch
streams, integer handles or None (the current torch stream when torch is
loaded, else the legacy default stream).

A C pointer carries neither its memory space nor its length, so for tensors
and NumPy arrays the binding checks what the library cannot: the buffer is
contiguous, lives where the entry point expects it (device memory for the
device entry points, host memory for fmmfft_translate_host) and holds at
least the bytes the plan's extents address.  A failed check raises
FmmfftError(FMMFFT_ERR_INVALID_ARG) before anything is launched.  Integer
addresses are passed through as given, unchecked.

Importing the package does not load the library; the first call does, and it
raises if libfmmfft.so is missing (build it with
``python -m paper_2010_00520_gb300.build``).  There is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfmmfft.so")

FMMFFT_OK = 0
FMMFFT_ERR_INVALID_ARG = -1
FMMFFT_ERR_NOT_COMPRESSED = -2
FMMFFT_ERR_OOM = -3
FMMFFT_ERR_CUDA = -4
FMMFFT_ERR_UNSUPPORTED = -5
FMMFFT_ERR_DEVICE = -6
FMMFFT_ERR_IO = -7
FMMFFT_ERR_TOO_LARGE = -8
FMMFFT_NOALLOC_SCRATCH_BYTES = 32 << 20

FMMFFT_FORMAT_NONE, FMMFFT_FORMAT_3D, FMMFFT_FORMAT_4D = 0, 3, 4
FMMFFT_DECOMP_NONE, FMMFFT_DECOMP_TUCKER, FMMFFT_DECOMP_TT, FMMFFT_DECOMP_HTUCKER = 0, 1, 2, 3
FMMFFT_PREC_C128, FMMFFT_PREC_C64, FMMFFT_PREC_C64_3XTF32, FMMFFT_PREC_C64_BF16X3 = 0, 1, 2, 3
FMMFFT_PREC_C64_TF32 = 4
FMMFFT_KEY_PRECISION = 1
FMMFFT_KEY_NPHI_RULE = 2
FMMFFT_KEY_NEAR_RULE = 3
FMMFFT_KEY_KAPPA = 4
FMMFFT_KEY_PREFACTOR = 5
FMMFFT_KEY_TRUNC_RULE = 6
FMMFFT_KEY_PROFILE = 7
FMMFFT_KEY_EPS_R_RE = 8
FMMFFT_KEY_EPS_R_IM = 9
FMMFFT_KEY_HOST_BLOCKS = 10
FMMFFT_KEY_DIR_FIRST = 11
FMMFFT_KEY_DIR_COUNT = 12
FMMFFT_KEY_RESTORE_ERROR = 13
FMMFFT_STAGE_RESTORE, FMMFFT_STAGE_XFWD, FMMFFT_STAGE_YZ, FMMFFT_STAGE_XINV = 0, 1, 2, 3
FMMFFT_NUM_STAGES = 4

# every symbol the header declares
EXPORTED = (
    "fmmfft_plan_create", "fmmfft_plan_set", "fmmfft_compress", "fmmfft_import_plain",
    "fmmfft_import_tucker3d", "fmmfft_translate", "fmmfft_translate_host", "fmmfft_plan_stats",
    "fmmfft_plan_directions", "fmmfft_poll_status", "fmmfft_plan_destroy", "fmmfft_status_string",
    "fmmfft_operator_host", "fmmfft_compress_direction_host", "fmmfft_stage_times",
    "fmmfft_plan_ranks", "fmmfft_translate_noalloc", "fmmfft_import_tt3d", "fmmfft_import_tucker4d",
    "fmmfft_import_htucker", "fmmfft_import_tt4d", "fmmfft_compress_host",
    "fmmfft_batch_create", "fmmfft_batch_translate", "fmmfft_batch_destroy", "fmmfft_plan_save",
    "fmmfft_plan_load", "fmmfft_autotune", "fmmfft_batch_autotune", "fmmfft_multipole_count",
    "fmmfft_aggregate", "fmmfft_disaggregate", "fmmfft_translate_disaggregate", "fmmfft_plan_set_occupancy",
    "fmmfft_batch_shared_count",
)


class FmmfftError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {fmmfft_status_string(status)} ({status})")


class _Stats(ctypes.Structure):
    _fields_ = [
        ("n_dir", ctypes.c_int), ("L", ctypes.c_int), ("K", ctypes.c_int * 3), ("n", ctypes.c_int * 3),
        ("format", ctypes.c_int), ("decomp", ctypes.c_int), ("precision", ctypes.c_int),
        ("max_rank", ctypes.c_int * 6), ("mean_rank", ctypes.c_double * 3),
        ("elements_plain", ctypes.c_int64), ("elements_compressed", ctypes.c_int64),
        ("saving", ctypes.c_double), ("device_bytes_operator", ctypes.c_int64),
        ("device_bytes_scratch", ctypes.c_int64), ("setup_seconds", ctypes.c_double),
        ("restore_on_tensor_cores", ctypes.c_int), ("kernel_launches", ctypes.c_int),
        ("large_planes", ctypes.c_int), ("schedule", ctypes.c_int * 4),
        ("restore_rel_err", ctypes.c_double),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libfmmfft.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2010_00520_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "fmmfft_plan_create": [ctypes.POINTER(vp), i, i, i, d, d, i, i, i, d],
        "fmmfft_plan_set": [vp, i, d],
        "fmmfft_compress": [vp],
        "fmmfft_import_plain": [vp, dp],
        "fmmfft_import_tucker3d": [vp, ip, dp, dp, dp, dp],
        "fmmfft_import_tt3d": [vp, ip, dp, dp, dp],
        "fmmfft_import_tucker4d": [vp, ip, dp, dp, dp, dp, dp],
        "fmmfft_import_htucker": [vp, ip, dp, dp, dp, dp, dp, dp, dp],
        "fmmfft_import_tt4d": [vp, ip, dp, dp, dp, dp],
        "fmmfft_compress_host": [vp, ip, dp],
        "fmmfft_batch_create": [ctypes.POINTER(vp), ctypes.POINTER(vp), i],
        "fmmfft_batch_translate": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ip, vp],
        "fmmfft_batch_destroy": [vp],
        "fmmfft_plan_save": [vp, ctypes.c_char_p],
        "fmmfft_autotune": [vp, i, d],
        "fmmfft_batch_autotune": [vp, ip, d],
        "fmmfft_plan_load": [ctypes.POINTER(vp), ctypes.c_char_p],
        "fmmfft_translate": [vp, vp, vp, i, vp],
        "fmmfft_translate_host": [vp, vp, vp, i, vp],
        "fmmfft_translate_noalloc": [vp, vp, vp, i, vp],
        "fmmfft_plan_stats": [vp, ctypes.POINTER(_Stats)],
        "fmmfft_plan_directions": [vp, dp, dp],
        "fmmfft_poll_status": [vp, ip],
        "fmmfft_plan_destroy": [vp],
        "fmmfft_status_string": [i],
        "fmmfft_operator_host": [vp, i, dp],
        "fmmfft_compress_direction_host": [vp, i, ip, dp],
        "fmmfft_stage_times": [vp, ctypes.POINTER(ctypes.c_float)],
        "fmmfft_plan_ranks": [vp, ip],
        "fmmfft_multipole_count": [d, d, d, d, d, ip],
        "fmmfft_aggregate": [vp, vp, vp, vp, i, i, vp],
        "fmmfft_disaggregate": [vp, vp, vp, vp, i, i, vp],
        "fmmfft_translate_disaggregate": [vp, vp, vp, vp, i, i, vp],
        "fmmfft_plan_set_occupancy": [vp, vp],
        "fmmfft_batch_shared_count": [vp, ip],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "fmmfft_status_string" else ctypes.c_int
    _lib = L
    return L


def _check(st: int, where: str):
    if st != FMMFFT_OK:
        raise FmmfftError(st, where)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _extents(plan):
    """(directions, boxes per field, bytes per complex element) of `plan`."""
    s = _Stats()
    _check(lib().fmmfft_plan_stats(plan, ctypes.byref(s)), "fmmfft_plan_stats")
    return s.n_dir, s.K[0] * s.K[1] * s.K[2], 16 if s.precision == FMMFFT_PREC_C128 else 8


def _sized(*bufs) -> bool:
    """True when any buffer is an object whose size the binding can check."""
    return any(b is not None and not isinstance(b, int) for b in bufs)


def _buffer(x, device: bool, need, where: str, what: str) -> int:
    """Address of one field, pattern or coefficient buffer after the checks a
    bare pointer cannot carry.  A torch tensor or NumPy array must be
    contiguous, in device memory for a device entry point (a kernel given a
    host address faults, or on a GPU that reaches host memory reads the wrong
    data) or in host memory for the host entry point, and hold at least
    `need` bytes (None: not checked) -- the kernels address the full extents
    of the plan.  None and integer addresses pass through unchecked."""
    if x is None or isinstance(x, int):
        return _ptr(x)
    if isinstance(x, np.ndarray):
        on_device, contiguous, nbytes = False, bool(x.flags.c_contiguous), int(x.nbytes)
    elif hasattr(x, "is_cuda") and hasattr(x, "numel") and hasattr(x, "element_size"):
        on_device = bool(x.is_cuda)
        contiguous = bool(x.is_contiguous())
        nbytes = int(x.numel()) * int(x.element_size())
    else:
        return _ptr(x)
    if on_device != device:
        raise FmmfftError(FMMFFT_ERR_INVALID_ARG,
                          f"{where}: {what} is in {'device' if on_device else 'host'} memory, "
                          f"this entry point takes {'device' if device else 'host'} memory")
    if not contiguous:
        raise FmmfftError(FMMFFT_ERR_INVALID_ARG, f"{where}: {what} is not contiguous")
    if need is not None and nbytes < need:
        raise FmmfftError(FMMFFT_ERR_INVALID_ARG,
                          f"{where}: {what} holds {nbytes} bytes, the plan's extents need {need}")
    return _ptr(x)


def _fields(plan, S_in, S_out, nrhs, device: bool, where: str, tag: str = ""):
    """Checked addresses of the input and output fields [n_dir][2][nrhs][Kz][Ky][Kx]
    (plan None: memory space and layout only)."""
    need = None
    if plan is not None and nrhs >= 1 and _sized(S_in, S_out):
        nd, V, es = _extents(plan)
        need = nd * 2 * nrhs * V * es
    return (_buffer(S_in, device, need, where, "S_in" + tag), _buffer(S_out, device, need, where, "S_out" + tag))


def _far_field(plan, patterns, per_box, spectra, nb, nrhs, where: str, names):
    """Checked addresses of the far-field buffers: patterns [n_dir][2][nb][V],
    the per-box coefficients or results [nrhs][nb][V] and the spectra
    [n_dir][2][nrhs][V]."""
    need = (None, None, None)
    if nb >= 1 and nrhs >= 1 and _sized(patterns, per_box, spectra):
        nd, V, es = _extents(plan)
        need = (nd * 2 * nb * V * es, nrhs * nb * V * es, nd * 2 * nrhs * V * es)
    return tuple(_buffer(b, True, n, where, w) for b, n, w in zip((patterns, per_box, spectra), need, names))


def _stream(s) -> int:
    if s is None:
        import sys
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
        return 0
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError(f"unsupported stream {type(s)}")


def _cplx(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def fmmfft_status_string(status: int) -> str:
    return lib().fmmfft_status_string(int(status)).decode()


def fmmfft_plan_create(Nx, Ny, Nz, a, k0, L, format, decomp, tol) -> int:
    h = ctypes.c_void_p()
    _check(lib().fmmfft_plan_create(ctypes.byref(h), Nx, Ny, Nz, float(a), float(k0), L, format, decomp,
                                    float(tol)), "fmmfft_plan_create")
    return h.value


def fmmfft_plan_set(plan, key, value):
    _check(lib().fmmfft_plan_set(plan, key, float(value)), "fmmfft_plan_set")


def fmmfft_compress(plan):
    _check(lib().fmmfft_compress(plan), "fmmfft_compress")


def _import_ranks(plan, ranks, per_dir: int, count: int, where: str):
    """Rank array of an import (int32, contiguous) and the plan's (n, n_dir).
    The library reads `count` ranks (per direction for the 3D formats) and,
    from them, the lengths of the factor arrays; a short rank array would be
    read past its end, so it is refused here."""
    st = fmmfft_plan_stats(plan)
    r = np.ascontiguousarray(ranks, dtype=np.int32).ravel()
    need = count * (st["n_dir"] if per_dir else 1)
    if r.size < need:
        raise FmmfftError(FMMFFT_ERR_INVALID_ARG, f"{where}: {r.size} ranks given, the plan needs {need}")
    return r, tuple(st["n"]), st["n_dir"]


def _import_arrays(where: str, ranks, named_arrays, needs):
    """Contiguous complex128 copies of the factor arrays, each checked to hold
    at least the complex values its ranks imply (the library reads exactly
    that many).  Ranks below 1 are left to the library to refuse."""
    arrs = [_cplx(x) for _, x in named_arrays]
    if np.all(np.asarray(ranks) >= 1):
        for (name, _), a, n in zip(named_arrays, arrs, needs):
            if a.size < n:
                raise FmmfftError(FMMFFT_ERR_INVALID_ARG,
                                  f"{where}: {name} holds {a.size} complex values, the ranks need {n}")
    return arrs


def fmmfft_import_plain(plan, That):
    st = fmmfft_plan_stats(plan)
    n = st["n"]
    T, = _import_arrays("fmmfft_import_plain", [1], [("That", That)], [st["n_dir"] * n[0] * n[1] * n[2]])
    _check(lib().fmmfft_import_plain(plan, _dptr(T)), "fmmfft_import_plain")


def fmmfft_import_tucker3d(plan, ranks, core, U1, U2, U3):
    where = "fmmfft_import_tucker3d"
    r, n, nd = _import_ranks(plan, ranks, True, 3, where)
    rd = r[:3 * nd].reshape(nd, 3).astype(np.int64)
    needs = [int(np.prod(rd, axis=1).sum())] + [n[i] * int(rd[:, i].sum()) for i in range(3)]
    arrs = _import_arrays(where, rd, [("core", core), ("U1", U1), ("U2", U2), ("U3", U3)], needs)
    _check(lib().fmmfft_import_tucker3d(plan, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        *[_dptr(x) for x in arrs]), where)


def _ints(x):
    r = np.ascontiguousarray(x, dtype=np.int32)
    return r, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def fmmfft_import_tt3d(plan, ranks, U1, C1, U3):
    where = "fmmfft_import_tt3d"
    r, n, nd = _import_ranks(plan, ranks, True, 2, where)
    rd = r[:2 * nd].reshape(nd, 2).astype(np.int64)
    needs = [n[0] * int(rd[:, 0].sum()), n[1] * int((rd[:, 0] * rd[:, 1]).sum()), n[2] * int(rd[:, 1].sum())]
    arrs = _import_arrays(where, rd, [("U1", U1), ("C1", C1), ("U3", U3)], needs)
    _check(lib().fmmfft_import_tt3d(plan, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                    *[_dptr(x) for x in arrs]), where)


def fmmfft_import_tucker4d(plan, ranks, core, U1, U2, U3, U4):
    where = "fmmfft_import_tucker4d"
    r, n, nd = _import_ranks(plan, ranks, False, 4, where)
    q = [int(v) for v in r[:4]]
    dims = (n[0], n[1], n[2], nd)
    needs = [q[0] * q[1] * q[2] * q[3]] + [dims[i] * q[i] for i in range(4)]
    arrs = _import_arrays(where, q, [("core", core), ("U1", U1), ("U2", U2), ("U3", U3), ("U4", U4)], needs)
    _check(lib().fmmfft_import_tucker4d(plan, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        *[_dptr(x) for x in arrs]), where)


def fmmfft_import_htucker(plan, ranks, U1, U2, U3, U4, C12, C34, B):
    where = "fmmfft_import_htucker"
    r, n, nd = _import_ranks(plan, ranks, False, 6, where)
    q = [int(v) for v in r[:6]]
    dims = (n[0], n[1], n[2], nd)
    needs = [dims[i] * q[i] for i in range(4)] + [q[0] * q[1] * q[4], q[2] * q[3] * q[5], q[4] * q[5]]
    named = [("U1", U1), ("U2", U2), ("U3", U3), ("U4", U4), ("C12", C12), ("C34", C34), ("B", B)]
    arrs = _import_arrays(where, q, named, needs)
    _check(lib().fmmfft_import_htucker(plan, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                       *[_dptr(x) for x in arrs]), where)


def fmmfft_import_tt4d(plan, ranks, U1, C1, C2, U3):
    where = "fmmfft_import_tt4d"
    r, n, nd = _import_ranks(plan, ranks, False, 3, where)
    q = [int(v) for v in r[:3]]
    needs = [n[0] * q[0], q[0] * n[1] * q[1], q[1] * n[2] * q[2], nd * q[2]]
    arrs = _import_arrays(where, q, [("U1", U1), ("C1", C1), ("C2", C2), ("U3", U3)], needs)
    _check(lib().fmmfft_import_tt4d(plan, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                    *[_dptr(x) for x in arrs]), where)


def fmmfft_compress_host(plan, restored=True):
    """Host FP64 compression of the whole operator in the plan's format:
    returns (ranks, restored) with ranks an (n_dir, 3) array for 3D formats or
    6 ints for 4D formats, restored (n_dir, n1, n2, n3) or None."""
    st = fmmfft_plan_stats(plan)
    nd, n = st["n_dir"], tuple(st["n"])
    is3d = st["format"] == FMMFFT_FORMAT_3D
    r = np.zeros(nd * 3 if is3d else 6, dtype=np.int32)
    out = np.zeros((nd,) + n, dtype=np.complex128) if restored else None
    _check(lib().fmmfft_compress_host(plan, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      _dptr(out) if restored else None), "fmmfft_compress_host")
    return (r.reshape(nd, 3) if is3d else r), out


def fmmfft_autotune(plan, nrhs, budget_ms=2000.0):
    _check(lib().fmmfft_autotune(plan, int(nrhs), float(budget_ms)), "fmmfft_autotune")


def fmmfft_batch_autotune(batch, nrhs, budget_ms=2000.0):
    r, rp = _ints(nrhs)
    plans = _BATCH_PLANS.get(batch)
    if plans is not None and r.size != len(plans):
        raise FmmfftError(FMMFFT_ERR_INVALID_ARG,
                          f"fmmfft_batch_autotune: {r.size} RHS counts for a batch of {len(plans)} plans")
    _check(lib().fmmfft_batch_autotune(batch, rp, float(budget_ms)), "fmmfft_batch_autotune")


def fmmfft_plan_save(plan, path):
    _check(lib().fmmfft_plan_save(plan, os.fsencode(path)), "fmmfft_plan_save")


def fmmfft_plan_load(path) -> int:
    h = ctypes.c_void_p()
    _check(lib().fmmfft_plan_load(ctypes.byref(h), os.fsencode(path)), "fmmfft_plan_load")
    return h.value


# The plans of each batch made through this binding.  The library reads one
# entry of S_in, S_out and nrhs per plan of the batch, from C arrays that
# carry no length, so the lists' lengths (and each instance's buffers) are
# checked against these.
_BATCH_PLANS: dict = {}


def fmmfft_batch_create(plans) -> int:
    plans = list(plans)
    arr = (ctypes.c_void_p * len(plans))(*plans)
    h = ctypes.c_void_p()
    _check(lib().fmmfft_batch_create(ctypes.byref(h), arr, len(plans)), "fmmfft_batch_create")
    _BATCH_PLANS[h.value] = plans
    return h.value


def fmmfft_batch_translate(batch, S_in, S_out, nrhs, stream=None):
    where = "fmmfft_batch_translate"
    r, rp = _ints(nrhs)
    plans = _BATCH_PLANS.get(batch)
    n = len(S_in)
    if not (len(S_out) == r.size == n) or (plans is not None and n != len(plans)):
        raise FmmfftError(FMMFFT_ERR_INVALID_ARG,
                          f"{where}: {n} inputs, {len(S_out)} outputs and {r.size} RHS counts"
                          + (f" for a batch of {len(plans)} plans" if plans is not None else ""))
    pairs = [_fields(plans[i] if plans is not None else None, S_in[i], S_out[i], int(r.flat[i]), True,
                     where, f"[{i}]") for i in range(n)]
    ins = (ctypes.c_void_p * n)(*[a for a, _ in pairs])
    outs = (ctypes.c_void_p * n)(*[b for _, b in pairs])
    _check(lib().fmmfft_batch_translate(batch, ins, outs, rp, _stream(stream)), where)


def fmmfft_batch_destroy(batch):
    _check(lib().fmmfft_batch_destroy(batch), "fmmfft_batch_destroy")
    _BATCH_PLANS.pop(batch, None)


def fmmfft_translate(plan, S_in, S_out, nrhs, stream=None):
    i, o = _fields(plan, S_in, S_out, int(nrhs), True, "fmmfft_translate")
    _check(lib().fmmfft_translate(plan, i, o, int(nrhs), _stream(stream)), "fmmfft_translate")


def fmmfft_aggregate(plan, patterns, currents, A, nb, nrhs, stream=None):
    """Eq. 4 on the device: A[p][c][r][v] = sum_i P[p][c][i][v] I[r][i][v]."""
    p, c, a = _far_field(plan, patterns, currents, A, int(nb), int(nrhs), "fmmfft_aggregate",
                         ("patterns", "currents", "A"))
    _check(lib().fmmfft_aggregate(plan, p, c, a, int(nb), int(nrhs), _stream(stream)), "fmmfft_aggregate")


def fmmfft_disaggregate(plan, patterns, B, y, nb, nrhs, stream=None):
    """Eq. 6 on the device: y[r][i][v] = sum_p w_p sum_c conj(P[p][c][i][v]) B[p][c][r][v]."""
    p, o, b = _far_field(plan, patterns, y, B, int(nb), int(nrhs), "fmmfft_disaggregate",
                         ("patterns", "y", "B"))
    _check(lib().fmmfft_disaggregate(plan, p, b, o, int(nb), int(nrhs), _stream(stream)), "fmmfft_disaggregate")


def fmmfft_translate_disaggregate(plan, S_in, patterns, y, nb, nrhs, stream=None):
    """Eq. 5 then Eq. 6 on the device, the translated fields kept on chip:
    y[r][i][v] = sum_p w_p sum_c conj(P[p][c][i][v]) B[p][c][r][v] with
    B the translation of S_in."""
    p, o, b = _far_field(plan, patterns, y, S_in, int(nb), int(nrhs), "fmmfft_translate_disaggregate",
                         ("patterns", "y", "S_in"))
    _check(lib().fmmfft_translate_disaggregate(plan, b, p, o, int(nb), int(nrhs), _stream(stream)),
           "fmmfft_translate_disaggregate")


def fmmfft_batch_shared_count(batch) -> int:
    """Instances of the last batch call that ran in the shared launches (one
    per phase and shape class)."""
    n = ctypes.c_int()
    _check(lib().fmmfft_batch_shared_count(batch, ctypes.byref(n)), "fmmfft_batch_shared_count")
    return n.value


def fmmfft_plan_set_occupancy(plan, occupied=None):
    """Box occupancy mask (Kz, Ky, Kx) of the plan's grid, nonzero = occupied
    (Sec. II.A: empty boxes carry no sources and receive nothing), or None to
    clear it."""
    if occupied is None:
        _check(lib().fmmfft_plan_set_occupancy(plan, None), "fmmfft_plan_set_occupancy")
        return
    st = fmmfft_plan_stats(plan)
    Kx, Ky, Kz = st["K"]
    m = np.ascontiguousarray(np.asarray(occupied) != 0, dtype=np.uint8)
    if m.size != Kx * Ky * Kz:
        raise FmmfftError(FMMFFT_ERR_INVALID_ARG,
                          f"fmmfft_plan_set_occupancy: mask of {m.size} boxes for a grid of {Kx * Ky * Kz}")
    _check(lib().fmmfft_plan_set_occupancy(plan, m.ctypes.data_as(ctypes.c_void_p)), "fmmfft_plan_set_occupancy")


def fmmfft_translate_noalloc(plan, S_in, S_out, nrhs, stream=None):
    """fmmfft_translate without any device allocation: the intermediate lives
    in the library's fixed 32 MiB device array (shared by every call; order
    calls on one stream).  Raises FmmfftError(FMMFFT_ERR_TOO_LARGE) when the
    workload's intermediate does not fit."""
    i, o = _fields(plan, S_in, S_out, int(nrhs), True, "fmmfft_translate_noalloc")
    _check(lib().fmmfft_translate_noalloc(plan, i, o, int(nrhs), _stream(stream)), "fmmfft_translate_noalloc")


def fmmfft_translate_host(plan, S_in, S_out, nrhs, stream=None):
    i, o = _fields(plan, S_in, S_out, int(nrhs), False, "fmmfft_translate_host")
    _check(lib().fmmfft_translate_host(plan, i, o, int(nrhs), _stream(stream)), "fmmfft_translate_host")


def fmmfft_plan_stats(plan) -> dict:
    s = _Stats()
    _check(lib().fmmfft_plan_stats(plan, ctypes.byref(s)), "fmmfft_plan_stats")
    out = {}
    for name, _ in _Stats._fields_:
        v = getattr(s, name)
        out[name] = list(v) if isinstance(v, ctypes.Array) else v
    return out


def fmmfft_plan_ranks(plan):
    n = fmmfft_plan_stats(plan)["n_dir"]
    r = np.zeros((n, 3), dtype=np.int32)
    _check(lib().fmmfft_plan_ranks(plan, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "fmmfft_plan_ranks")
    return r


def fmmfft_plan_directions(plan):
    n = fmmfft_plan_stats(plan)["n_dir"]
    kh = np.zeros((n, 3))
    w = np.zeros(n)
    _check(lib().fmmfft_plan_directions(plan, _dptr(kh), _dptr(w)), "fmmfft_plan_directions")
    return kh, w


def fmmfft_operator_host(plan, p):
    st = fmmfft_plan_stats(plan)
    out = np.zeros(tuple(st["n"]), dtype=np.complex128)
    _check(lib().fmmfft_operator_host(plan, int(p), _dptr(out)), "fmmfft_operator_host")
    return out


def fmmfft_compress_direction_host(plan, p, restored=True):
    st = fmmfft_plan_stats(plan)
    r = np.zeros(3, dtype=np.int32)
    out = np.zeros(tuple(st["n"]), dtype=np.complex128) if restored else None
    _check(lib().fmmfft_compress_direction_host(plan, int(p), r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                _dptr(out) if restored else None),
           "fmmfft_compress_direction_host")
    return tuple(int(v) for v in r), out


def fmmfft_stage_times(plan):
    ms = (ctypes.c_float * FMMFFT_NUM_STAGES)()
    _check(lib().fmmfft_stage_times(plan, ms), "fmmfft_stage_times")
    return [float(v) for v in ms]


def fmmfft_poll_status(plan) -> int:
    v = ctypes.c_int(0)
    _check(lib().fmmfft_poll_status(plan, ctypes.byref(v)), "fmmfft_poll_status")
    return v.value


def fmmfft_multipole_count(a, k0, digits, eps_r=1.0):
    """L of the excess-bandwidth rule (Sec. II.A) for boxes of edge a, free-space
    wavenumber k0, relative permittivity eps_r (complex, Im <= 0)."""
    e = complex(eps_r)
    L = ctypes.c_int(0)
    _check(lib().fmmfft_multipole_count(a, k0, e.real, e.imag, digits, ctypes.byref(L)), "fmmfft_multipole_count")
    return L.value


def fmmfft_plan_destroy(plan):
    _check(lib().fmmfft_plan_destroy(plan), "fmmfft_plan_destroy")


class Plan:
    """Owning wrapper around a plan handle (destroyed on close / exit)."""

    def __init__(self, K, a, k0, L, format=FMMFFT_FORMAT_NONE, decomp=FMMFFT_DECOMP_NONE, tol=0.0, **opts):
        self.handle = fmmfft_plan_create(K[0], K[1], K[2], a, k0, L, format, decomp, tol)
        keys = {"precision": FMMFFT_KEY_PRECISION, "nphi_rule": FMMFFT_KEY_NPHI_RULE,
                "near_rule": FMMFFT_KEY_NEAR_RULE, "kappa": FMMFFT_KEY_KAPPA,
                "prefactor": FMMFFT_KEY_PREFACTOR, "trunc_rule": FMMFFT_KEY_TRUNC_RULE,
                "profile": FMMFFT_KEY_PROFILE, "eps_r_re": FMMFFT_KEY_EPS_R_RE,
                "eps_r_im": FMMFFT_KEY_EPS_R_IM, "host_blocks": FMMFFT_KEY_HOST_BLOCKS,
                "dir_first": FMMFFT_KEY_DIR_FIRST, "dir_count": FMMFFT_KEY_DIR_COUNT,
                "restore_error": FMMFFT_KEY_RESTORE_ERROR}
        for k, v in opts.items():
            fmmfft_plan_set(self.handle, keys[k], v)

    def compress(self):
        fmmfft_compress(self.handle)
        return self

    def stats(self) -> dict:
        return fmmfft_plan_stats(self.handle)

    def translate(self, S_in, S_out, nrhs, stream=None):
        fmmfft_translate(self.handle, S_in, S_out, nrhs, stream)

    def close(self):
        if self.handle:
            fmmfft_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
