"""CPU tests of the binding's buffer checks.

A C pointer carries neither its memory space nor its length, so the binding
checks torch tensors and NumPy arrays before it hands their addresses to the
library: device memory for the device entry points, host memory for
fmmfft_translate_host, contiguous, and at least the bytes the plan's extents
address.  Each rejection must come from the binding (FMMFFT_ERR_INVALID_ARG)
where the library itself would have answered differently, and each accepted
call must reach the library.  Device buffers are stood in for by objects
with the attributes of a CUDA tensor whose addresses are never dereferenced:
every accepted call here is one the library refuses on the host (an
uncompressed plan, an unsupported basis-function count)."""
import numpy as np
import pytest

TWO_PI = 2 * np.pi


class DeviceBuffer:
    """Stands in for a contiguous CUDA tensor of `nbytes` bytes."""

    def __init__(self, nbytes, contiguous=True, addr=1 << 40):
        self.is_cuda = True
        self._n = nbytes // 8
        self._contiguous = contiguous
        self._addr = addr

    def data_ptr(self):
        return self._addr

    def numel(self):
        return self._n

    def element_size(self):
        return 8

    def is_contiguous(self):
        return self._contiguous


def _status(fn, *args):
    import paper_2010_00520_gb300 as F
    with pytest.raises(F.FmmfftError) as e:
        fn(*args)
    return e.value.status


@pytest.fixture
def plan(native):
    F = native
    K, L = (4, 5, 3), 2
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, 0, 0, 0.0)
    yield F, h, F.fmmfft_plan_stats(h)["n_dir"], K[0] * K[1] * K[2]
    F.fmmfft_plan_destroy(h)


def test_device_entry_points_take_device_buffers_of_the_plans_size(plan):
    torch = pytest.importorskip("torch")
    F, h, nd, V = plan
    for nrhs in (1, 3):
        need = nd * 2 * nrhs * V * 8
        ok = DeviceBuffer(need)
        # accepted by the binding, refused by the library (not compressed)
        for fn in (F.fmmfft_translate, F.fmmfft_translate_noalloc):
            assert _status(fn, h, ok, DeviceBuffer(need, addr=2 << 40), nrhs, 0) == F.FMMFFT_ERR_NOT_COMPRESSED
        bad = [
            (DeviceBuffer(need - 8), DeviceBuffer(need, addr=2 << 40)),               # input one element short
            (ok, DeviceBuffer(need - 8, addr=2 << 40)),                               # output one element short
            (ok, DeviceBuffer(need, contiguous=False, addr=2 << 40)),                 # strided
            (torch.zeros(need // 8, dtype=torch.complex64), DeviceBuffer(need, addr=2 << 40)),  # host tensor
            (ok, np.zeros(need // 8, dtype=np.complex64)),                            # NumPy (host) array
        ]
        for fn in (F.fmmfft_translate, F.fmmfft_translate_noalloc):
            for x, y in bad:
                assert _status(fn, h, x, y, nrhs, 0) == F.FMMFFT_ERR_INVALID_ARG
    # bare addresses are not checked: the library answers
    assert _status(F.fmmfft_translate, h, 1 << 40, 2 << 40, 1, 0) == F.FMMFFT_ERR_NOT_COMPRESSED
    # an invalid RHS count is left to the library as well
    assert _status(F.fmmfft_translate, h, DeviceBuffer(8), DeviceBuffer(8, addr=2 << 40), 0, 0) == \
        F.FMMFFT_ERR_NOT_COMPRESSED


def test_complex128_plans_need_twice_the_bytes(plan):
    F, h, nd, V = plan
    F.fmmfft_plan_set(h, F.FMMFFT_KEY_PRECISION, F.FMMFFT_PREC_C128)
    need = nd * 2 * V * 16
    assert _status(F.fmmfft_translate, h, DeviceBuffer(need), DeviceBuffer(need, addr=2 << 40), 1, 0) == \
        F.FMMFFT_ERR_NOT_COMPRESSED
    assert _status(F.fmmfft_translate, h, DeviceBuffer(need // 2), DeviceBuffer(need, addr=2 << 40), 1, 0) == \
        F.FMMFFT_ERR_INVALID_ARG


def test_host_entry_point_takes_host_buffers(plan):
    torch = pytest.importorskip("torch")
    F, h, nd, V = plan
    nrhs = 2
    n = nd * 2 * nrhs * V
    x, y = np.zeros(n, dtype=np.complex64), np.zeros(n, dtype=np.complex64)
    assert _status(F.fmmfft_translate_host, h, x, y, nrhs, 0) == F.FMMFFT_ERR_NOT_COMPRESSED
    assert _status(F.fmmfft_translate_host, h, torch.zeros(n, dtype=torch.complex64),
                   torch.zeros(n, dtype=torch.complex64), nrhs, 0) == F.FMMFFT_ERR_NOT_COMPRESSED
    assert _status(F.fmmfft_translate_host, h, x[:-1], y, nrhs, 0) == F.FMMFFT_ERR_INVALID_ARG
    assert _status(F.fmmfft_translate_host, h, x, DeviceBuffer(n * 8), nrhs, 0) == F.FMMFFT_ERR_INVALID_ARG
    z = np.zeros(2 * n, dtype=np.complex64)[::2]
    assert _status(F.fmmfft_translate_host, h, z, y, nrhs, 0) == F.FMMFFT_ERR_INVALID_ARG


def test_far_field_buffers_are_checked_per_role(plan):
    """Patterns [n_dir][2][nb][V], per-box coefficients or results
    [nrhs][nb][V], spectra [n_dir][2][nrhs][V]: each role has its own size.
    nb = 49 is above the kernels' limit, so a call the binding accepts comes
    back from the library as FMMFFT_ERR_UNSUPPORTED."""
    F, h, nd, V = plan
    nb, nrhs = 49, 2
    sizes = {"P": nd * 2 * nb * V * 8, "box": nrhs * nb * V * 8, "spec": nd * 2 * nrhs * V * 8}
    base = {k: DeviceBuffer(v, addr=(i + 1) << 40) for i, (k, v) in enumerate(sizes.items())}
    agg = lambda b: (F.fmmfft_aggregate, h, b["P"], b["box"], b["spec"], nb, nrhs, 0)
    dis = lambda b: (F.fmmfft_disaggregate, h, b["P"], b["spec"], b["box"], nb, nrhs, 0)
    for call in (agg, dis):
        assert _status(*call(base)) == F.FMMFFT_ERR_UNSUPPORTED
        for role in sizes:
            short = dict(base, **{role: DeviceBuffer(sizes[role] - 8, addr=7 << 40)})
            assert _status(*call(short)) == F.FMMFFT_ERR_INVALID_ARG, role
        host = dict(base, P=np.zeros(sizes["P"] // 8, dtype=np.complex64))
        assert _status(*call(host)) == F.FMMFFT_ERR_INVALID_ARG


def test_batch_takes_device_buffers(native):
    """The batch handle does not expose its plans, so the batch call checks
    the memory space and layout of each buffer, not its size; the check runs
    before the library sees the (here null) handle."""
    torch = pytest.importorskip("torch")
    F = native
    cases = [([torch.zeros(8, dtype=torch.complex64)], [DeviceBuffer(64)], "S_in[0] is in host memory"),
             ([DeviceBuffer(64)], [np.zeros(8, dtype=np.complex64)], "S_out[0] is in host memory"),
             ([DeviceBuffer(64), DeviceBuffer(64, contiguous=False)], [DeviceBuffer(64)] * 2,
              "S_in[1] is not contiguous")]
    for ins, outs, msg in cases:
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_batch_translate(0, ins, outs, [1] * len(ins), 0)
        assert e.value.status == F.FMMFFT_ERR_INVALID_ARG and msg in str(e.value)
    # device buffers pass: the library then refuses the null handle
    with pytest.raises(F.FmmfftError) as e:
        F.fmmfft_batch_translate(0, [DeviceBuffer(64)], [DeviceBuffer(64, addr=2 << 40)], [1], 0)
    assert e.value.status == F.FMMFFT_ERR_INVALID_ARG and "memory" not in str(e.value)


def _oracle_parts(K, L, fmt, dec, tol):
    from oracle import pipeline as pl
    plan = pl.Plan(K=K, L=L)
    ops = pl.operators(plan)
    return ops, pl.compress(ops, fmt, dec, tol).parts


def _import_args(F, fmt, dec, P, short=None):
    """The import call of one format with the oracle's factors, laid out as
    the library's header states; `short` names one array to cut by one value."""
    cat = lambda xs: np.concatenate([np.ravel(x) for x in xs])
    if fmt == "3d" and dec == "tucker":
        fn, ranks = F.fmmfft_import_tucker3d, np.array([t.ranks for t in P], dtype=np.int32)
        named = [("core", cat([t.core for t in P]))] + \
                [(f"U{i + 1}", cat([t.factors[i] for t in P])) for i in range(3)]
    elif fmt == "3d":
        fn, ranks = F.fmmfft_import_tt3d, np.array([t.ranks for t in P], dtype=np.int32)
        named = [("U1", cat([t.U1 for t in P])), ("C1", cat([t.cores[0] for t in P])),
                 ("U3", cat([t.Ud for t in P]))]
    elif dec == "tucker":
        fn, ranks = F.fmmfft_import_tucker4d, np.array(P.ranks, dtype=np.int32)
        named = [("core", P.core)] + [(f"U{i + 1}", u) for i, u in enumerate(P.factors)]
    elif dec == "htucker":
        fn, ranks = F.fmmfft_import_htucker, np.array(P.ranks, dtype=np.int32)
        named = [(f"U{i + 1}", u) for i, u in enumerate(P.U)] + [("C12", P.C12), ("C34", P.C34), ("B", P.B)]
    else:
        fn, ranks = F.fmmfft_import_tt4d, np.array(P.ranks, dtype=np.int32)
        named = [("U1", P.U1), ("C1", P.cores[0]), ("C2", P.cores[1]), ("U3", P.Ud)]
    arrays = [np.ravel(a)[:-1] if name == short else a for name, a in named]
    return fn, ranks, arrays, [name for name, _ in named]


def _import_status(fn, h, *args):
    """0 when the import succeeds (a machine with a device), else its status."""
    import paper_2010_00520_gb300 as F
    try:
        fn(h, *args)
        return 0
    except F.FmmfftError as e:
        return e.status


FORMATS = [("3d", "tucker", 3, 1), ("3d", "tt", 3, 2), ("4d", "tucker", 4, 1), ("4d", "htucker", 4, 3),
           ("4d", "tt", 4, 2)]


@pytest.mark.parametrize("fmt,dec,cfmt,cdec", FORMATS)
def test_imports_take_the_oracles_factors_and_refuse_short_arrays(native, fmt, dec, cfmt, cdec):
    """The oracle's factors pass the binding's length checks and reach the
    library, whose host-side checks accept them too (on a machine without a
    device the upload then fails with a status other than
    FMMFFT_ERR_INVALID_ARG); every factor array one value short, and a short
    rank array, is refused before the library reads it."""
    F = native
    K, L, tol = (6, 5, 7), 2, 1e-3
    _, P = _oracle_parts(K, L, fmt, dec, tol)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, cfmt, cdec, tol)
    try:
        fn, ranks, arrays, names = _import_args(F, fmt, dec, P)
        assert _import_status(fn, h, ranks, *arrays) != F.FMMFFT_ERR_INVALID_ARG
        for name in names:
            fn, ranks, arrays, _ = _import_args(F, fmt, dec, P, short=name)
            with pytest.raises(F.FmmfftError) as e:
                fn(h, ranks, *arrays)
            assert e.value.status == F.FMMFFT_ERR_INVALID_ARG and f"{name} holds" in str(e.value), name
        fn, ranks, arrays, _ = _import_args(F, fmt, dec, P)
        with pytest.raises(F.FmmfftError) as e:
            fn(h, np.ravel(ranks)[:-1], *arrays)
        assert e.value.status == F.FMMFFT_ERR_INVALID_ARG and "ranks given" in str(e.value)
    finally:
        F.fmmfft_plan_destroy(h)


def test_plain_import_takes_the_whole_operator(native):
    F = native
    K, L = (6, 5, 7), 2
    ops, _ = _oracle_parts(K, L, "3d", "tucker", 1e-3)
    h = F.fmmfft_plan_create(*K, 0.5, TWO_PI, L, 0, 0, 0.0)
    try:
        assert _import_status(F.fmmfft_import_plain, h, np.stack(ops)) != F.FMMFFT_ERR_INVALID_ARG
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_import_plain(h, np.stack(ops[:-1]))
        assert e.value.status == F.FMMFFT_ERR_INVALID_ARG and "That holds" in str(e.value)
    finally:
        F.fmmfft_plan_destroy(h)


def test_batch_lists_match_the_batch(native, plan):
    """The library reads one S_in, S_out and nrhs entry per plan of the batch;
    the binding checks the lists against the plans it recorded at batch
    creation and each instance's buffers against its plan.  A batch needs
    compressed plans, so the recorded plans are set here for the null handle,
    which the library itself refuses once the binding lets a call through."""
    F, h, nd, V = plan
    need = nd * 2 * 2 * V * 8
    ok = [DeviceBuffer(need)], [DeviceBuffer(need, addr=2 << 40)]

    def message(ins, outs, nrhs):
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_batch_translate(0, ins, outs, nrhs, 0)
        assert e.value.status == F.FMMFFT_ERR_INVALID_ARG
        return str(e.value)

    assert "2 inputs, 1 outputs" in message(ok[0] * 2, ok[1], [2, 2])
    F._BATCH_PLANS[0] = [h]
    try:
        assert "for a batch of 1 plans" in message(ok[0] * 2, ok[1] * 2, [2, 2])
        assert "S_in[0] holds" in message([DeviceBuffer(need - 8)], ok[1], [2])
        assert "holds" not in message(ok[0], ok[1], [2])           # reaches the library
        with pytest.raises(F.FmmfftError) as e:
            F.fmmfft_batch_autotune(0, [1, 2], 10.0)
        assert "2 RHS counts for a batch of 1 plans" in str(e.value)
    finally:
        F._BATCH_PLANS.pop(0, None)
