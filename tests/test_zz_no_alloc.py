"""The allocation-free SpMV entry point.

Some callers may not allocate device memory when they need a product: a
real-time loop whose memory is fixed before it starts, or a framework that
owns all device memory.  spx_spmv_csr_noalloc serves them from one fixed
scratch array.  Here it is checked against the CPU oracle and against the
ordinary handle-based spx_spmv on two calls in a row (the fixed array keeps
the previous call's contents), and its size limit is checked.  This file is
named to run last."""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import TOL, assert_spmv_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def spx():
    from paper_2103_10116_gb300 import spx as s
    s.load()
    return s


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("which", ["stencil27", "powerlaw"])
def test_no_alloc_matches_oracle_and_spmv(spx, which, dtype):
    if which == "stencil27":
        rp, col, val = synth.stencil3d_27pt(30)
    else:  # long rows: exercises the cross-tile look-back
        rp, col, val = synth.powerlaw(60000, mean=16, max_len=6000, seed=5)
    n = rp.shape[0] - 1
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    rp_d, col_d, val_d = t(rp), t(col), t(val).to(dtype)
    key = "f64" if dtype == torch.float64 else "f32"
    vr = val.astype(np.float32).astype(np.float64) if key == "f32" else val
    ctx = spx.spx_ctx_create(0)
    A = spx.spx_matrix_create(ctx, "csr", rp_d, col_d, val_d)
    try:
        for seed in (1, 2):  # two calls in a row on the same fixed array
            xh = synth.uniform_vector(n, seed)
            xr = xh.astype(np.float32).astype(np.float64) if key == "f32" else xh
            x = t(xh).to(dtype)
            y = torch.full((n,), float("nan"), dtype=dtype, device=DEV)
            spx.spx_spmv_csr_noalloc(rp_d, col_d, val_d, x, y)
            y_spmv = torch.empty(n, dtype=dtype, device=DEV)
            spx.spx_spmv(ctx, A, x, y_spmv)
            torch.cuda.synchronize()
            yn = y.double().cpu().numpy()
            assert np.isfinite(yn).all()  # a bounded wait that gave up would leave NaN
            y_orc = oracle.spmv_csr(rp, col, vr, xr)
            bound = oracle.spmv_absbound(rp, col, vr, xr)
            assert_spmv_close(yn, y_orc, bound, TOL[key])
            assert_spmv_close(yn, y_spmv.double().cpu().numpy(), bound, TOL[key])
    finally:
        spx.spx_matrix_destroy(A)
        spx.spx_ctx_destroy(ctx)


def test_no_alloc_rejects_sizes_beyond_its_scratch(spx):
    fn = spx.load().spx_spmv_csr_noalloc
    # nrows + nnz beyond 32768 tiles of 2048 items: refused before any device work
    rc = fn(None, spx.SPX_F64, 40_000_000, 40_000_000, 40_000_000, 16, 16, 16, 16, 16)
    assert rc == spx.SPX_ERR_TOO_LARGE
    assert "scratch limit" in spx.spx_last_error()
