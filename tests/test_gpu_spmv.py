"""GPU parity of every SpMV kernel and format against the CPU oracle, and
byte-exact checks of the device format conversions.  Calls go through the C
ABI (ctypes binding)."""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import TOL, assert_spmv_close, random_int_csr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def spx():
    from paper_2103_10116_gb300 import spx as s
    s.load()
    return s


@pytest.fixture(scope="module")
def ctx(spx):
    c = spx.spx_ctx_create(0)
    yield c
    torch.cuda.synchronize()
    spx.spx_ctx_destroy(c)


def _long_row_matrix():
    # many empty rows, one very long row (spans several merge / COO tiles),
    # ragged short rows, duplicates and unsorted columns
    rng = np.random.default_rng(7)
    n = 9000
    lens = np.zeros(n, np.int64)
    lens[0] = 7000
    lens[1:50] = rng.integers(0, 9, size=49)
    lens[3001:] = rng.integers(0, 5, size=n - 3001)
    lens[8999] = 3000
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(lens)
    col = rng.integers(0, n, size=int(rp[-1])).astype(np.int32)
    val = rng.standard_normal(int(rp[-1]))
    return rp, col, val


def _rect_matrix():
    rng = np.random.default_rng(11)
    rp, col, val = random_int_csr(rng, 3000, 1700, max_len=40, empty_frac=0.3)
    return rp, col, val.astype(np.float64) * 0.731


MATRICES = {
    "lap2d_64": lambda: synth.laplace2d_5pt(64),
    "st27_23": lambda: synth.stencil3d_27pt(23),
    "powerlaw_60k": lambda: synth.powerlaw(60000, mean=16, max_len=6000, seed=5),
    "convdiff_20": lambda: synth.convdiff3d_upwind(20),
    "longrow": _long_row_matrix,
    "rect": _rect_matrix,
    "tiny1": lambda: (np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5])),
    "empty_rows": lambda: (np.zeros(40, np.int32), np.zeros(0, np.int32), np.zeros(0)),
}

VARIANTS = [
    ("csr", None, 0),
    ("csr", "vector", 1), ("csr", "vector", 4), ("csr", "vector", 32),
    ("csr", "merge", 4), ("csr", "merge", 8), ("csr", "merge", 16),
    ("csr", "split", 8), ("csr", "split", 16), ("csr", "tiled", 16), ("csr", "tiled", 32), ("csr", "rows", 0), ("csr", "rows", 1), ("csr", "rows", 22),
    ("csr", "rows", 42),
    ("ell", None, 0), ("ell", "ell", 1),
    ("coo", None, 0), ("coo", "coo", 1), ("coo", "coo", 8), ("coo", "coo", 16), ("coo", "coo", 216),
    ("coo", "coo", 232), ("coo", "coo", 104), ("coo", "coo", 116),
    ("hyb", None, 0), ("hyb0", None, 0), ("hyb3", None, 0), ("hyb3", "coo", 232),
]

_cache = {}


def _mat(name):
    if name not in _cache:
        rp, col, val = MATRICES[name]()
        ncols = int(col.max()) + 1 if name == "rect" and col.size else rp.shape[0] - 1
        if name == "rect":
            ncols = 1700
        x = synth.uniform_vector(ncols, seed=1)
        _cache[name] = (rp, col, val, ncols, x)
    return _cache[name]


def _make(spx, ctx, fmt, rp, col, val, ncols, dtype, flags=0):
    hyb_width = -1
    f = fmt
    if fmt.startswith("hyb") and fmt != "hyb":
        hyb_width = int(fmt[3:])
        f = "hyb"
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return spx.spx_matrix_create(ctx, f, t(rp), t(col), t(val).to(dtype), ncols=ncols, hyb_width=hyb_width,
                                 flags=flags)


def _kernel_code(spx, kname):
    return {None: spx.SPX_KERNEL_AUTO, "vector": spx.SPX_KERNEL_CSR_VECTOR, "merge": spx.SPX_KERNEL_CSR_MERGE,
            "split": spx.SPX_KERNEL_CSR_SPLIT, "rows": spx.SPX_KERNEL_CSR_ROWS, "tiled": spx.SPX_KERNEL_CSR_TILED,
            "ell": spx.SPX_KERNEL_ELL, "coo": spx.SPX_KERNEL_COO}[kname]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: f"{v[0]}-{v[1]}-{v[2]}")
@pytest.mark.parametrize("mname", list(MATRICES))
def test_spmv_parity(spx, ctx, mname, variant, dtype):
    fmt, kname, param = variant
    rp, col, val, ncols, x = _mat(mname)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":  # reference: FP64 oracle on the FP32-rounded inputs
        val_r, x_r = val.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64)
    else:
        val_r, x_r = val, x
    A = _make(spx, ctx, fmt, rp, col, val, ncols, tdt)
    try:
        if kname is not None:
            spx.spx_matrix_set_kernel(A, _kernel_code(spx, kname), param)
        n = rp.shape[0] - 1
        xd = torch.from_numpy(x).to(DEV).to(tdt)
        y = torch.full((n,), float("nan"), dtype=tdt, device=DEV)
        try:
            spx.spx_spmv(ctx, A, xd, y)
        except spx.SpxError as err:
            # the row-block kernels hold a tile of 128 rows in shared memory; a
            # matrix whose tile does not fit is rejected, never computed wrongly
            if (kname == "rows" or (kname, param) == ("coo", 1)) and err.status == spx.SPX_ERR_TOO_LARGE:
                pytest.skip("tile of 128 rows does not fit in shared memory")
            raise
        torch.cuda.synchronize()
        yref = oracle.spmv_csr(rp, col, val_r, x_r)
        bound = oracle.spmv_absbound(rp, col, val_r, x_r)
        assert_spmv_close(y.double().cpu().numpy(), yref, bound, TOL[dtype])
        # run-to-run determinism: identical bits
        y2 = torch.empty_like(y)
        spx.spx_spmv(ctx, A, xd, y2)
        torch.cuda.synchronize()
        assert torch.equal(y, y2)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo", "hyb"])
def test_spmv_axpby_and_host(spx, ctx, fmt):
    rp, col, val, ncols, x = _mat("powerlaw_60k")
    A = _make(spx, ctx, fmt, rp, col, val, ncols, torch.float64)
    try:
        n = rp.shape[0] - 1
        z = synth.uniform_vector(n, seed=9)
        y = torch.from_numpy(z).to(DEV)
        spx.spx_spmv_axpby(ctx, A, -1.5, torch.from_numpy(x).to(DEV), 0.25, y)
        torch.cuda.synchronize()
        ax = oracle.spmv_csr(rp, col, val, x)
        ref = -1.5 * ax + 0.25 * z
        bound = 1.5 * oracle.spmv_absbound(rp, col, val, x) + 0.25 * np.abs(z)
        assert_spmv_close(y.cpu().numpy(), ref, bound, 1e-12)
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty(n, dtype=torch.float64).pin_memory()
        spx.spx_spmv_host(ctx, A, xh, yh)
        assert_spmv_close(yh.numpy(), ax, oracle.spmv_absbound(rp, col, val, x), 1e-12)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("mname", ["lap2d_64", "powerlaw_60k", "longrow", "rect", "tiny1", "empty_rows"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_conversions_bit_exact(spx, ctx, mname, dtype):
    rp, col, val, ncols, _ = _mat(mname)
    npdt = np.float64 if dtype == "f64" else np.float32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    v = val.astype(npdt)
    n = rp.shape[0] - 1
    # CSR keeps the arrays as given
    A = _make(spx, ctx, "csr", rp, col, v, ncols, tdt)
    try:
        assert np.array_equal(spx.spx_matrix_export(ctx, A, spx.SPX_PART_ROW_PTR).cpu().numpy(), rp)
        assert np.array_equal(spx.spx_matrix_export(ctx, A, spx.SPX_PART_COL).cpu().numpy(), col)
        assert spx.spx_matrix_export(ctx, A, spx.SPX_PART_VAL).cpu().numpy().tobytes() == v.tobytes()
    finally:
        spx.spx_matrix_destroy(A)
    # COO
    A = _make(spx, ctx, "coo", rp, col, v, ncols, tdt)
    try:
        assert np.array_equal(spx.spx_matrix_export(ctx, A, spx.SPX_PART_COO_ROW).cpu().numpy(),
                              oracle.csr_to_coo_rows(rp))
        assert np.array_equal(spx.spx_matrix_export(ctx, A, spx.SPX_PART_COO_COL).cpu().numpy(), col)
        assert spx.spx_matrix_export(ctx, A, spx.SPX_PART_COO_VAL).cpu().numpy().tobytes() == v.tobytes()
    finally:
        spx.spx_matrix_destroy(A)
    # ELL (skip when the padded width would be huge for the test)
    if oracle.max_row_len(rp) * max(n, 1) <= 80_000_000:
        A = _make(spx, ctx, "ell", rp, col, v, ncols, tdt)
        try:
            info = spx.spx_matrix_get_info(A)
            w, ld = info["ell_width"], info["ell_ld"]
            assert w == oracle.max_row_len(rp) and ld % 32 == 0 and ld >= n
            ec, ev = oracle.csr_to_ell(rp, col, v, w, ld)
            assert np.array_equal(spx.spx_matrix_export(ctx, A, spx.SPX_PART_ELL_COL).cpu().numpy(), ec)
            assert spx.spx_matrix_export(ctx, A, spx.SPX_PART_ELL_VAL).cpu().numpy().tobytes() == ev.tobytes()
        finally:
            spx.spx_matrix_destroy(A)
    # HYB: auto width and fixed widths
    for hw in (-1, 0, 3):
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
        A = spx.spx_matrix_create(ctx, "hyb", t(rp), t(col), t(v), ncols=ncols, hyb_width=hw)
        try:
            info = spx.spx_matrix_get_info(A)
            w, ld = info["ell_width"], info["ell_ld"]
            want_w = oracle.hyb_auto_width(rp, v.itemsize) if hw < 0 else min(hw, oracle.max_row_len(rp))
            assert w == want_w
            ec, ev, cr, cc, cv = oracle.csr_to_hyb(rp, col, v, w, ld)
            assert info["coo_nnz"] == cr.shape[0]
            assert np.array_equal(spx.spx_matrix_export(ctx, A, spx.SPX_PART_ELL_COL).cpu().numpy(), ec)
            assert spx.spx_matrix_export(ctx, A, spx.SPX_PART_ELL_VAL).cpu().numpy().tobytes() == ev.tobytes()
            if cr.shape[0]:
                assert np.array_equal(spx.spx_matrix_export(ctx, A, spx.SPX_PART_COO_ROW).cpu().numpy(), cr)
                assert np.array_equal(spx.spx_matrix_export(ctx, A, spx.SPX_PART_COO_COL).cpu().numpy(), cc)
                assert spx.spx_matrix_export(ctx, A, spx.SPX_PART_COO_VAL).cpu().numpy().tobytes() == cv.tobytes()
        finally:
            spx.spx_matrix_destroy(A)


def test_mixed_shadow_is_fp32_rounding(spx, ctx):
    rp, col, val, ncols, _ = _mat("st27_23")
    A = _make(spx, ctx, "csr", rp, col, val * 1.37, ncols, torch.float64, flags=spx.SPX_MIXED_SHADOW)
    try:
        s = spx.spx_matrix_export(ctx, A, spx.SPX_PART_VAL_F32).cpu().numpy()
        assert s.tobytes() == (val * 1.37).astype(np.float32).tobytes()
        assert spx.spx_matrix_get_info(A)["has_f32_shadow"] == 1
    finally:
        spx.spx_matrix_destroy(A)


def test_invalid_csr_is_rejected(spx, ctx):
    t = lambda a: torch.tensor(a, dtype=torch.int32, device=DEV)
    v = torch.ones(3, dtype=torch.float64, device=DEV)
    for rp, col in ([[0, 2, 1, 3], [0, 1, 2]],      # decreasing row pointer
                    [[1, 2, 3, 3], [0, 1, 2]],      # rp[0] != 0
                    [[0, 1, 2, 3], [0, 5, 2]],      # column out of range
                    [[0, 1, 2, 3], [0, -1, 2]]):    # negative column
        with pytest.raises(spx.SpxError) as ei:
            spx.spx_matrix_create(ctx, "csr", t(rp), t(col), v)
        assert ei.value.status == spx.SPX_ERR_INVALID


def test_ell_of_a_huge_row_is_too_large(spx, ctx):
    n = 2_000_000
    rp = torch.zeros(n + 1, dtype=torch.int32)
    rp[1:] = n
    col = torch.arange(n, dtype=torch.int32)
    val = torch.ones(n, dtype=torch.float64)
    with pytest.raises(spx.SpxError) as ei:
        spx.spx_matrix_create(ctx, "ell", rp.to(DEV), col.to(DEV), val.to(DEV))
    assert ei.value.status == spx.SPX_ERR_TOO_LARGE
    # the same matrix is fine as HYB / CSR
    A = spx.spx_matrix_create(ctx, "hyb", rp.to(DEV), col.to(DEV), val.to(DEV))
    spx.spx_matrix_destroy(A)


def test_host_input_flag(spx, ctx):
    rp, col, val, ncols, x = _mat("lap2d_64")
    A = spx.spx_matrix_create(ctx, "csr", torch.from_numpy(rp), torch.from_numpy(col), torch.from_numpy(val))
    try:
        y = torch.empty(rp.shape[0] - 1, dtype=torch.float64, device=DEV)
        spx.spx_spmv(ctx, A, torch.from_numpy(x).to(DEV), y)
        torch.cuda.synchronize()
        assert_spmv_close(y.cpu().numpy(), oracle.spmv_csr(rp, col, val, x), oracle.spmv_absbound(rp, col, val, x),
                          TOL["f64"])
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_dot_and_axpby(spx, ctx, dtype):
    n = 1_234_567
    a = torch.from_numpy(synth.uniform_vector(n, 1)).to(DEV).to(dtype)
    b = torch.from_numpy(synth.uniform_vector(n, 2)).to(DEV).to(dtype)
    r = torch.empty(1, dtype=dtype, device=DEV)
    spx.spx_dot(ctx, a, b, r)
    r2 = torch.empty(1, dtype=dtype, device=DEV)
    spx.spx_dot(ctx, a, b, r2)
    torch.cuda.synchronize()
    ref = float(np.dot(a.double().cpu().numpy(), b.double().cpu().numpy()))
    bound = float(np.dot(np.abs(a.double().cpu().numpy()), np.abs(b.double().cpu().numpy())))
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert abs(float(r) - ref) <= tol * bound
    assert torch.equal(r, r2)
    y = b.clone()
    spx.spx_axpby(ctx, 2.0, a, -0.5, y)
    torch.cuda.synchronize()
    ref = 2.0 * a.double() - 0.5 * b.double()
    assert torch.allclose(y.double(), ref, rtol=tol, atol=tol)


def test_rows_kernel_tile_too_large(spx, ctx):
    """The row-block kernel holds a tile of 128 rows in shared memory: a matrix
    with a 60,000-entry row cannot use it (SPX_ERR_TOO_LARGE, nothing
    launched), and the automatic choice falls back to another kernel."""
    n = 300
    lens = np.full(n, 3, np.int64)
    lens[7] = 60000
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(lens)
    rng = np.random.default_rng(3)
    col = rng.integers(0, n, size=int(rp[-1])).astype(np.int32)
    val = rng.standard_normal(int(rp[-1]))
    x = synth.uniform_vector(n, seed=2)
    A = _make(spx, ctx, "csr", rp, col, val, n, torch.float64)
    try:
        xd = torch.from_numpy(x).to(DEV)
        y = torch.empty(n, dtype=torch.float64, device=DEV)
        spx.spx_matrix_set_kernel(A, spx.SPX_KERNEL_CSR_ROWS, 0)
        with pytest.raises(spx.SpxError) as ei:
            spx.spx_spmv(ctx, A, xd, y)
        assert ei.value.status == spx.SPX_ERR_TOO_LARGE
        spx.spx_matrix_set_kernel(A, spx.SPX_KERNEL_AUTO, 0)
        spx.spx_spmv(ctx, A, xd, y)
        torch.cuda.synchronize()
        yref = oracle.spmv_csr(rp, col, val, x)
        assert_spmv_close(y.cpu().numpy(), yref, oracle.spmv_absbound(rp, col, val, x), TOL["f64"])
    finally:
        spx.spx_matrix_destroy(A)


def test_gather_probe_runs_and_checks_arguments(spx, ctx):
    """The gather-floor measurement aid streams the pattern and stores nothing."""
    n, nnz = 5000, 120000
    rng = np.random.default_rng(9)
    col = torch.from_numpy(rng.integers(0, n, size=nnz).astype(np.int32)).to(DEV)
    for tdt in (torch.float64, torch.float32):
        x = torch.from_numpy(rng.uniform(-1, 1, n)).to(DEV).to(tdt)
        out = torch.zeros(1, dtype=tdt, device=DEV)
        spx.spx_probe_gather(ctx, col, x, out)
        torch.cuda.synchronize()
        assert float(out[0]) == 0.0
    with pytest.raises((spx.SpxError, TypeError)):  # integer x: rejected before or by the library
        spx.spx_probe_gather(ctx, col, torch.zeros(n, dtype=torch.int32, device=DEV), out)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("mname,fmt", [("st27_23", "csr"), ("powerlaw_60k", "csr"), ("longrow", "csr"),
                                       ("st27_23", "ell"), ("powerlaw_60k", "coo"), ("powerlaw_60k", "hyb")])
def test_tune_keeps_a_correct_kernel(spx, ctx, mname, fmt, dtype, tmp_path):
    """The autotuner times every variant (skipping those that do not fit, e.g.
    the row-block kernels on the long-row matrix), keeps the fastest, and the
    kept kernel computes the product correctly; the JSON cache replays it."""
    rp, col, val, ncols, x = _mat(mname)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    val_r, x_r = (val.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64)) \
        if dtype == "f32" else (val, x)
    A = _make(spx, ctx, fmt, rp, col, val, ncols, tdt)
    try:
        k, p, us = spx.spx_matrix_tune(ctx, A, reps=3)
        info = spx.spx_matrix_get_info(A)
        assert (info["kernel"], info["kernel_param"]) == (k, p) and us > 0
        n = rp.shape[0] - 1
        y = torch.full((n,), float("nan"), dtype=tdt, device=DEV)
        spx.spx_spmv(ctx, A, torch.from_numpy(x).to(DEV).to(tdt), y)
        torch.cuda.synchronize()
        assert_spmv_close(y.double().cpu().numpy(), oracle.spmv_csr(rp, col, val_r, x_r),
                          oracle.spmv_absbound(rp, col, val_r, x_r), TOL[dtype])
        path = str(tmp_path / "tune.json")
        k1, p1, us1 = spx.tune_cached(ctx, A, path, reps=3)
        spx.spx_matrix_set_kernel(A, spx.SPX_KERNEL_AUTO, 0)
        assert spx.tune_cached(ctx, A, path) == (k1, p1, None) and us1 is not None
        info = spx.spx_matrix_get_info(A)
        assert (info["kernel"], info["kernel_param"]) == (k1, p1)
    finally:
        spx.spx_matrix_destroy(A)


def test_tune_rejects_bad_reps(spx, ctx):
    rp, col, val, ncols, x = _mat("lap2d_64")
    A = _make(spx, ctx, "csr", rp, col, val, ncols, torch.float64)
    try:
        with pytest.raises(spx.SpxError) as ei:
            spx.spx_matrix_tune(ctx, A, reps=0)
        assert ei.value.status == spx.SPX_ERR_INVALID
    finally:
        spx.spx_matrix_destroy(A)
