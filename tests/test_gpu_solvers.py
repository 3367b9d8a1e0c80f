"""GPU Krylov solvers against the CPU oracle: convergence to the stated
tolerance on the TRUE residual (re-formed here by the oracle's SpMV on the
GPU's x), error against the manufactured solution x*, iteration counts close
to the oracle's, and the edge cases (b = 0, max_iter, initial guess, fixed
iteration mode)."""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import residual_limit

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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _true_relres(rp, col, val, b, x):
    r = b - oracle.spmv_csr(rp, col, val, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


def _problem(name):
    if name == "lap2d_64":
        rp, col, val = synth.laplace2d_5pt(64)
    elif name == "lap3d_20":
        rp, col, val = synth.laplace3d_7pt(20)
    elif name == "convdiff_16":
        rp, col, val = synth.convdiff3d_upwind(16)
    elif name == "convdiff_12":
        rp, col, val = synth.convdiff3d_upwind(12)
    else:
        raise KeyError(name)
    n = rp.shape[0] - 1
    xs = synth.uniform_vector(n, seed=3)
    b = oracle.spmv_csr(rp, col, val, xs)
    return rp, col, val, xs, b


def _make(spx, ctx, fmt, rp, col, val, flags=0, kernel=None, param=0, dtype=torch.float64):
    A = spx.spx_matrix_create(ctx, fmt, _t(rp), _t(col), _t(val).to(dtype), flags=flags)
    if kernel is not None:
        spx.spx_matrix_set_kernel(A, kernel, param)
    return A


def _fmt_kernel(spx, fmt):
    """'csr-rowsP' names the row-block CSR kernel with parameter P; returns (format, kernel, param)."""
    if fmt.startswith("csr-rows"):
        return "csr", spx.SPX_KERNEL_CSR_ROWS, int(fmt[8:])
    if fmt.startswith("csr-tiled"):
        return "csr", spx.SPX_KERNEL_CSR_TILED, int(fmt[9:])
    if fmt.startswith("coo-tiled"):
        return "coo", spx.SPX_KERNEL_COO, int(fmt[9:])
    return fmt, None, 0


FMTS = [("csr", None, 0), ("csr", 1, 4), ("csr", 2, 16), ("csr", 5, 16), ("csr", 7, 16), ("csr", 7, 32),
        ("coo", 4, 232),
        ("csr", 6, 0), ("csr", 6, 22),
        ("csr", 6, 42), ("ell", None, 0),
        ("coo", None, 0), ("hyb", None, 0)]


@pytest.mark.parametrize("fmt", FMTS, ids=lambda f: f"{f[0]}-{f[1]}-{f[2]}")
def test_cg_laplace2d_64(spx, ctx, fmt):
    # the 64x64 5-point Laplacian, b = A x*, CG to 1e-10
    rp, col, val, xs, b = _problem("lap2d_64")
    A = _make(spx, ctx, fmt[0], rp, col, val, kernel=fmt[1], param=fmt[2])
    try:
        x = torch.zeros_like(_t(b))
        info = spx.spx_solve(ctx, A, _t(b), x, "cg", 1e-10, 5000)
        xh = x.cpu().numpy()
        _, oinfo = oracle.cg(rp, col, val, b, tol=1e-10, maxit=5000)
        assert info.status == spx.SPX_CONVERGED, info
        assert info.relres_true <= 1e-10 and _true_relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, 1e-10)
        assert abs(info.iterations - oinfo.iterations) <= max(3, oinfo.iterations // 10), (info, oinfo)
        lam_min = 8 * np.sin(np.pi / 130) ** 2
        lam_max = 8 * np.cos(np.pi / 130) ** 2
        assert np.linalg.norm(xh - xs) / np.linalg.norm(xs) <= (lam_max / lam_min) * 1e-10
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo", "hyb", "csr-rows22", "csr-rows42", "csr-tiled32",
                                 "coo-tiled232"])
def test_bicgstab_convdiff(spx, ctx, fmt):
    rp, col, val, xs, b = _problem("convdiff_16")
    f, kernel, param = _fmt_kernel(spx, fmt)
    A = _make(spx, ctx, f, rp, col, val, kernel=kernel, param=param)
    try:
        x = torch.zeros_like(_t(b))
        info = spx.spx_solve(ctx, A, _t(b), x, "bicgstab", 1e-10, 5000)
        _, oinfo = oracle.bicgstab(rp, col, val, b, tol=1e-10, maxit=5000)
        xh = x.cpu().numpy()
        assert info.status == spx.SPX_CONVERGED, info
        assert info.relres_true <= 1e-10 and _true_relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, 1e-10)
        assert abs(info.iterations - oinfo.iterations) <= max(3, oinfo.iterations // 10), (info, oinfo)
        assert np.linalg.norm(xh - xs) / np.linalg.norm(xs) <= 1e-7
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo", "hyb", "csr-rows22", "csr-rows42", "csr-tiled32"])
def test_cgs_convdiff(spx, ctx, fmt):
    rp, col, val, xs, b = _problem("convdiff_16")
    f, kernel, param = _fmt_kernel(spx, fmt)
    A = _make(spx, ctx, f, rp, col, val, kernel=kernel, param=param)
    try:
        x = torch.zeros_like(_t(b))
        info = spx.spx_solve(ctx, A, _t(b), x, "cgs", 1e-10, 5000)
        _, oinfo = oracle.cgs(rp, col, val, b, tol=1e-10, maxit=5000)
        xh = x.cpu().numpy()
        assert info.status == spx.SPX_CONVERGED, info
        assert info.relres_true <= 1e-10 and _true_relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, 1e-10)
        # CGS squares the residual polynomial: its convergence is irregular, rounding moves the stop
        assert abs(info.iterations - oinfo.iterations) <= max(4, oinfo.iterations // 5), (info, oinfo)
        assert np.linalg.norm(xh - xs) / np.linalg.norm(xs) <= 1e-7
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("c", [2.5, -1.5])
def test_cgs_scaled_identity_one_step(spx, ctx, c):
    n = 1000
    rp = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    val = np.full(n, c)
    b = synth.uniform_vector(n, seed=4)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, "cgs", 1e-12, 100)
        assert info.status == spx.SPX_CONVERGED and info.iterations == 1
        assert np.allclose(x.cpu().numpy(), b / c, rtol=1e-15, atol=0)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("fmt", ["csr", "csr-tiled32"])
@pytest.mark.parametrize("m", [5, 30])
def test_gmres_convdiff(spx, ctx, m, fmt):
    rp, col, val, xs, b = _problem("convdiff_12")
    f, kernel, param = _fmt_kernel(spx, fmt)
    A = _make(spx, ctx, f, rp, col, val, kernel=kernel, param=param)
    try:
        x = torch.zeros_like(_t(b))
        info = spx.spx_solve(ctx, A, _t(b), x, "gmres", 1e-10, 20000, restart=m)
        _, oinfo = oracle.gmres(rp, col, val, b, m=m, tol=1e-10, maxit=20000)
        xh = x.cpu().numpy()
        assert info.status == spx.SPX_CONVERGED, info
        assert info.relres_true <= 1e-10 and _true_relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, 1e-10)
        # CGS2 (GPU) and MGS (oracle) round differently: counts agree within 10% + a cycle's slack
        assert abs(info.iterations - oinfo.iterations) <= max(5, oinfo.iterations // 10), (info, oinfo)
    finally:
        spx.spx_matrix_destroy(A)


def test_gmres_minimal_polynomial(spx, ctx):
    n = 5000
    d = 6
    diag = np.linspace(1.0, 5.0, d)[np.arange(n) % d]
    rp = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    b = synth.uniform_vector(n, 1)
    A = _make(spx, ctx, "csr", rp, col, diag)
    try:
        x = torch.zeros_like(_t(b))
        info = spx.spx_solve(ctx, A, _t(b), x, "gmres", 1e-11, 100, restart=30)
        assert info.status == spx.SPX_CONVERGED and info.iterations <= d
        assert np.allclose(x.cpu().numpy(), b / diag, rtol=1e-9, atol=0)
    finally:
        spx.spx_matrix_destroy(A)


def test_cg_eigenvector_one_step(spx, ctx):
    m = 40
    rp, col, val = synth.laplace2d_5pt(m)
    iy, ix = np.meshgrid(np.arange(1, m + 1), np.arange(1, m + 1), indexing="ij")
    v = (np.sin(ix * 3 * np.pi / (m + 1)) * np.sin(iy * 2 * np.pi / (m + 1))).ravel()
    lam = 4 - 2 * np.cos(3 * np.pi / (m + 1)) - 2 * np.cos(2 * np.pi / (m + 1))
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(m * m, dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(v), x, "cg", 1e-12, 100)
        assert info.iterations == 1
        assert np.allclose(x.cpu().numpy(), v / lam, rtol=0, atol=1e-12)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver,prob", [("cg", "lap3d_20"), ("bicgstab", "convdiff_16"), ("cgs", "convdiff_16"),
                                         ("gmres", "convdiff_12")])
@pytest.mark.parametrize("fmt", ["csr", "ell", "hyb", "csr-tiled32", "coo-tiled232"])
def test_mixed_precision_ir(spx, ctx, solver, prob, fmt):
    rp, col, val, xs, b = _problem(prob)
    f, kernel, param = _fmt_kernel(spx, fmt)
    A = _make(spx, ctx, f, rp, col, val, flags=spx.SPX_MIXED_SHADOW, kernel=kernel, param=param)
    try:
        x = torch.zeros_like(_t(b))
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 20000, restart=30, precision="mixed")
        xh = x.cpu().numpy()
        assert info.status == spx.SPX_CONVERGED, info
        assert info.relres_true <= 1e-10 and _true_relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, 1e-10)
        assert info.restarts >= 2 and info.inner_iterations > 0
        assert np.linalg.norm(xh - xs) / np.linalg.norm(xs) <= 1e-7
        if solver == "cg":
            # CG: FP32 iterations with FP64 residual replacement (reliable updates)
            _, oinfo = oracle.cg_reliable(rp, col, val, b, tol=1e-10)
            assert oinfo.status == oracle.CONVERGED
            assert abs(info.iterations - oinfo.iterations) <= max(3, oinfo.iterations // 10), (info, oinfo)
            assert abs(info.restarts - oinfo.restarts) <= 3, (info, oinfo)
        elif solver != "gmres":
            _, oinfo = oracle.ir(rp, col, val, b, solver=solver, tol=1e-10)
            assert oinfo.status == oracle.CONVERGED
            assert abs(info.restarts - oinfo.restarts) <= 2, (info, oinfo)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_fp32_solve(spx, ctx, solver):
    rp, col, val, xs, b = _problem("lap3d_20")
    A = _make(spx, ctx, "csr", rp, col, val, dtype=torch.float32)
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float32, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b).float(), x, solver, 1e-5, 5000, precision="f32")
        assert info.status == spx.SPX_CONVERGED, info
        assert _true_relres(rp, col, val.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64),
                            x.double().cpu().numpy()) <= 2e-5
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_edge_cases(spx, ctx, solver):
    rp, col, val, xs, b = _problem("lap2d_64")
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        # b = 0 -> x = 0, zero iterations
        x = torch.ones(b.shape[0], dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, torch.zeros_like(x), x, solver, 1e-10, 100)
        assert info.status == spx.SPX_CONVERGED and info.iterations == 0 and float(x.abs().max()) == 0.0
        # max_iter reached -> status, not an error
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-14, 7)
        assert info.status == spx.SPX_MAX_ITER and info.iterations == 7
        # an initial guess is used: starting from x* converges at once
        x = _t(xs).clone()
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 100)
        assert info.status == spx.SPX_CONVERGED and info.iterations == 0
        # fixed-iteration mode runs exactly the requested count
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        info = spx.spx_solve_fixed(ctx, A, _t(b), x, solver, 40)
        assert info.iterations == 40
    finally:
        spx.spx_matrix_destroy(A)


def test_cg_full_size_poisson_128(spx, ctx):
    # the 128^3 7-point Poisson matrix (n = 2,097,152): CG to 1e-10 in the
    # configuration the benchmark uses; the true residual is re-formed on the CPU.
    rp, col, val = synth.laplace3d_7pt(128)
    n = rp.shape[0] - 1
    xs = synth.uniform_vector(n, seed=3)
    b = oracle.spmv_csr(rp, col, val, xs)
    A = _make(spx, ctx, "ell", rp, col, val)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, "cg", 1e-10, 5000)
        assert info.status == spx.SPX_CONVERGED, info
        assert _true_relres(rp, col, val, b, x.cpu().numpy()) <= residual_limit(rp, col, val, b, x.cpu().numpy(), 1e-10)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("n_side", [1, 3, 32, 64, 65, 100, 181])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_small_cg_single_launch_route(spx, ctx, n_side, dtype):
    """Small CSR systems with the automatic kernel: CG runs in one launch on a
    thread-block cluster (up to 32768 rows; n_side^2 rows here, from 1 row to
    32761, with slices of the cluster's blocks left empty or ragged).  Same
    oracle checks as the general path; FP32 to a tolerance it can reach."""
    rp, col, val = synth.laplace2d_5pt(n_side)
    n = rp.shape[0] - 1
    xs = synth.uniform_vector(n, seed=3)
    b = oracle.spmv_csr(rp, col, val, xs)
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    A = _make(spx, ctx, "csr", rp, col, val, dtype=dtype)
    try:
        x = torch.zeros(n, dtype=dtype, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b).to(dtype), x, "cg", tol, 20000,
                             precision="f64" if dtype == torch.float64 else "f32")
        assert info.status == spx.SPX_CONVERGED, info
        xh = x.double().cpu().numpy()
        _, oinfo = oracle.cg(rp, col, val, b, tol=tol, maxit=20000)
        if dtype == torch.float64:
            assert info.relres_true <= tol
            assert _true_relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, tol)
            assert abs(info.iterations - oinfo.iterations) <= max(3, oinfo.iterations // 10), (info, oinfo)
        else:  # FP32 arithmetic: the FP64 residual of the FP32 solution, with FP32 rounding slack
            assert _true_relres(rp, col, val, b, xh) <= 3 * tol
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs"])
def test_small_mixed_single_launch_route(spx, ctx, solver):
    """Mixed precision on a system of at most 4096 rows runs as a batch of one
    in the persistent batched kernel: CG with reliable updates, BiCGSTAB and
    CGS with refinement cycles, each against its oracle."""
    rp, col, val = synth.laplace2d_5pt(40) if solver == "cg" else synth.convdiff3d_upwind(12)
    n = rp.shape[0] - 1
    xs = synth.uniform_vector(n, seed=3)
    b = oracle.spmv_csr(rp, col, val, xs)
    A = _make(spx, ctx, "csr", rp, col, val, flags=spx.SPX_MIXED_SHADOW)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 20000, precision="mixed")
        assert info.status == spx.SPX_CONVERGED, info
        xh = x.cpu().numpy()
        assert _true_relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, 1e-10)
        if solver == "cg":
            _, oi = oracle.cg_reliable(rp, col, val, b, tol=1e-10)
            assert abs(info.iterations - oi.iterations) <= max(3, oi.iterations // 10), (info, oi)
            assert abs(info.restarts - oi.restarts) <= 3, (info, oi)
        else:
            _, oi = oracle.ir(rp, col, val, b, solver=solver, tol=1e-10)
            assert abs(info.restarts - oi.restarts) <= 2, (info, oi)
    finally:
        spx.spx_matrix_destroy(A)
