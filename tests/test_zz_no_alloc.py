"""The allocation-free SpMV entry point, for callers that cannot allocate
device memory when they need a product (graph capture, fixed-memory loops,
frameworks that own every allocation).  It must give what the ordinary
handle-based spx_spmv gives, on two calls in a row (the fixed scratch array
keeps the previous call's contents), and refuse sizes beyond its limit.
This file is named to run last."""
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
def test_no_alloc_matches_spmv(spx, which, dtype):
    if which == "stencil27":
        rp, col, val = synth.stencil3d_27pt(30)
    else:  # long rows: exercises the cross-tile look-back
        rp, col, val = synth.powerlaw(60000, mean=16, max_len=6000, seed=5)
    n = rp.shape[0] - 1
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    rp_d, col_d, val_d = t(rp), t(col), t(val).to(dtype)
    ctx = spx.spx_ctx_create(0)
    A = spx.spx_matrix_create(ctx, "csr", rp_d, col_d, val_d)
    spx.spx_matrix_set_kernel(A, spx.SPX_KERNEL_CSR_MERGE, 8)
    try:
        for seed in (1, 2):  # two calls in a row
            xh = synth.uniform_vector(n, seed)
            x = t(xh).to(dtype)
            y_ref = torch.empty(n, dtype=dtype, device=DEV)
            spx.spx_spmv(ctx, A, x, y_ref)
            y = torch.full((n,), float("nan"), dtype=dtype, device=DEV)
            spx.spx_spmv_csr_noalloc(rp_d, col_d, val_d, x, y)
            torch.cuda.synchronize()
            vr = val.astype(np.float32).astype(np.float64) if dtype == torch.float32 else val
            xr = xh.astype(np.float32).astype(np.float64) if dtype == torch.float32 else xh
            bound = oracle.spmv_absbound(rp, col, vr, xr)
            key = "f64" if dtype == torch.float64 else "f32"
            assert_spmv_close(y.double().cpu().numpy(), y_ref.double().cpu().numpy(), bound, TOL[key])
    finally:
        spx.spx_matrix_destroy(A)
        spx.spx_ctx_destroy(ctx)


def test_no_alloc_rejects_sizes_beyond_its_scratch(spx):
    limit = spx.load().spx_spmv_csr_noalloc
    # nrows + nnz beyond 32768 tiles of 2048 items: refused before any device work
    rc = limit(None, spx.SPX_F64, 40_000_000, 40_000_000, 40_000_000, 16, 16, 16, 16, 16)
    assert rc == spx.SPX_ERR_TOO_LARGE
    assert "scratch limit" in spx.spx_last_error()
