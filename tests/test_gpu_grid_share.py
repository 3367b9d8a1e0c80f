"""Launch grids sized for a share of the SMs (spx_ctx_set_grid_sms): every SpMV
kernel family and the Krylov solvers give the oracle's results with grids for
1, 8 and 38 SMs, and a matrix whose scratch was first sized by a narrow
context is then used by a whole-device context (buffers stay sized for the
device, so the wider grid fits)."""
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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def mats():
    pl = synth.powerlaw(200_000, seed=5)
    st = synth.stencil3d_27pt(30)
    return {"powerlaw": pl, "stencil": st}


# (format, kernel, param) for each kernel family; None = the format's default
KERNELS = [("csr", None, 0), ("csr", 2, 0), ("csr", 5, 8), ("csr", 6, 2), ("csr", 7, 32), ("ell", None, 0),
           ("coo", None, 0), ("coo", 4, 1), ("coo", 4, 8), ("hyb", None, 0)]


# ELL and the row-block CSR and COO kernels reject the power-law matrix as too large
CASES = [(m, f, k, p) for m in ("powerlaw", "stencil") for f, k, p in KERNELS
         if not (m == "powerlaw" and (f == "ell" or k == 6 or (f, k, p) == ("coo", 4, 1)))]


@pytest.mark.parametrize("share", [1, 8, 38])
@pytest.mark.parametrize("mname,fmt,kernel,param", CASES)
def test_spmv_with_narrow_grids(spx, mats, share, fmt, kernel, param, mname):
    rp, col, val = mats[mname]
    n = rp.shape[0] - 1
    x = synth.uniform_vector(n, seed=2)
    ctx = spx.spx_ctx_create(0)
    try:
        assert spx.spx_ctx_set_grid_sms(ctx, share) == share
        A = spx.spx_matrix_create(ctx, fmt, _t(rp), _t(col), _t(val))
        try:
            if kernel is not None:
                spx.spx_matrix_set_kernel(A, kernel, param)
            y = torch.empty(n, dtype=torch.float64, device=DEV)
            spx.spx_spmv(ctx, A, _t(x), y)
            spx.spx_ctx_check(ctx)
            ref = oracle.spmv_csr(rp, col, val, x)
            bound = oracle.spmv_absbound(rp, col, val, x)
            assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * bound + 1e-300)
        finally:
            spx.spx_matrix_destroy(A)
    finally:
        spx.spx_ctx_destroy(ctx)


@pytest.mark.parametrize("solver,prec", [("cg", "f64"), ("bicgstab", "f64"), ("gmres", "f64"), ("cg", "mixed"),
                                         ("cgs", "mixed")])
def test_solves_narrow_then_whole_device(spx, solver, prec):
    """A narrow context solves first (the matrix's workspace is created there),
    then a whole-device context solves the same matrix: both meet tol."""
    rp, col, val = synth.laplace3d_7pt(40) if solver == "cg" else synth.convdiff3d_upwind(32)
    n = rp.shape[0] - 1
    xs = synth.uniform_vector(n, seed=3)
    b = oracle.spmv_csr(rp, col, val, xs)
    narrow = spx.spx_ctx_create(0)
    wide = spx.spx_ctx_create(0)
    try:
        assert spx.spx_ctx_set_grid_sms(narrow, 4) == 4
        assert spx.spx_ctx_set_grid_sms(wide, 0) > 4
        A = spx.spx_matrix_create(narrow, "csr", _t(rp), _t(col), _t(val),
                                  flags=spx.SPX_MIXED_SHADOW if prec == "mixed" else 0)
        try:
            for c in (narrow, wide):
                x = torch.zeros(n, dtype=torch.float64, device=DEV)
                info = spx.spx_solve(c, A, _t(b), x, solver, 1e-10, 20000, restart=30, precision=prec)
                torch.cuda.synchronize()
                assert info.status == spx.SPX_CONVERGED, info
                xh = x.cpu().numpy()
                rel = np.linalg.norm(b - oracle.spmv_csr(rp, col, val, xh)) / np.linalg.norm(b)
                assert rel <= residual_limit(rp, col, val, b, xh, 1e-10)
        finally:
            spx.spx_matrix_destroy(A)
    finally:
        spx.spx_ctx_destroy(narrow)
        spx.spx_ctx_destroy(wide)


def test_grid_share_clamps(spx):
    ctx = spx.spx_ctx_create(0)
    try:
        full = spx.spx_ctx_set_grid_sms(ctx, 0)
        assert full == torch.cuda.get_device_properties(0).multi_processor_count
        assert spx.spx_ctx_set_grid_sms(ctx, 10 ** 6) == full
        assert spx.spx_ctx_set_grid_sms(ctx, -3) == full
        assert spx.spx_ctx_set_grid_sms(ctx, 5) == 5
    finally:
        spx.spx_ctx_destroy(ctx)
