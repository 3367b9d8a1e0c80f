"""Failure detection without a GPU fault: a device-side wait that nothing
satisfies (a look-back flag nobody publishes, an mbarrier phase nobody
completes) gives up after its limit, records the error, and the host sees
SPX_ERR_TIMEOUT from spx_ctx_check; the context stays usable (an SpMV right
after is correct) and a clean check follows."""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth

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


@pytest.mark.parametrize("which", [0, 1], ids=["lookback-flag", "mbarrier"])
def test_bounded_wait_reports_timeout_and_context_survives(spx, ctx, which):
    spx.spx_ctx_check(ctx)  # clean to start
    spx.spx_selftest_wait_timeout(ctx, which)
    with pytest.raises(spx.SpxError) as ei:
        spx.spx_ctx_check(ctx)
    assert ei.value.status == spx.SPX_ERR_TIMEOUT
    spx.spx_ctx_check(ctx)  # the error word was cleared
    rp, col, val = synth.laplace2d_5pt(32)
    x = synth.uniform_vector(32 * 32, seed=1)
    A = spx.spx_matrix_create(ctx, "csr", torch.from_numpy(rp).to(DEV), torch.from_numpy(col).to(DEV),
                              torch.from_numpy(val).to(DEV))
    try:
        y = torch.empty(32 * 32, dtype=torch.float64, device=DEV)
        spx.spx_spmv(ctx, A, torch.from_numpy(x).to(DEV), y)
        spx.spx_ctx_check(ctx)
        ref = oracle.spmv_csr(rp, col, val, x)
        assert np.allclose(y.cpu().numpy(), ref, rtol=1e-13, atol=1e-13)
    finally:
        spx.spx_matrix_destroy(A)


def test_selftest_rejects_bad_argument(spx, ctx):
    with pytest.raises(spx.SpxError) as ei:
        spx.spx_selftest_wait_timeout(ctx, 7)
    assert ei.value.status == spx.SPX_ERR_INVALID
