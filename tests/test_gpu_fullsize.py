"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (automatic kernel choice per format, the same seeded inputs):

* SpMV of the 27-point stencil on 100^3 (n = 1,000,000, nnz = 26,463,592) and of
  the power-law matrix (n = 2,000,000, nnz = 32,000,000) in every format and
  both value types, every row against the oracle's compensated SpMV;
* the 128^3 solves to 1e-10 (CG on the 7-point Poisson matrix, BiCGSTAB, CGS and
  GMRES(30) on the upwind convection-diffusion matrix), FP64 and FP32 inner +
  FP64 refinement: the true residual re-formed by the oracle, and the
  iteration counts of the oracle's CG / BiCGSTAB / CGS / GMRES(30) at full size;
* the 4096-system batch: a sample of systems checked one by one against the
  oracle (true residual, error, iteration count).
The oracle's arithmetic (plain C) takes tens of seconds here; no input or
expected value comes from the GPU path."""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import TOL, assert_spmv_close, residual_limit

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


_MATS = {}


def _mat(name):
    if name not in _MATS:
        _MATS[name] = {"stencil27_100": lambda: synth.stencil3d_27pt(100),
                       "powerlaw_2m": lambda: synth.powerlaw(2_000_000),
                       "poisson128": lambda: synth.laplace3d_7pt(128),
                       "convdiff128": lambda: synth.convdiff3d_upwind(128)}[name]()
    return _MATS[name]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


SWEEP = [("stencil27_100", f) for f in ("csr", "ell", "coo", "hyb")] + [("powerlaw_2m", f) for f in ("csr", "coo", "hyb")]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("mname,fmt", SWEEP, ids=lambda v: str(v))
def test_fullsize_spmv_every_row(spx, ctx, mname, fmt, dtype):
    rp, col, val = _mat(mname)
    n = rp.shape[0] - 1
    x = np.random.default_rng(1).uniform(-1, 1, n)  # the sweep's x
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":  # reference: the FP64 oracle on the FP32-rounded inputs
        val_r, x_r = val.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64)
    else:
        val_r, x_r = val, x
    A = spx.spx_matrix_create(ctx, fmt, _t(rp), _t(col), _t(val).to(tdt))
    try:
        y = torch.full((n,), float("nan"), dtype=tdt, device=DEV)
        spx.spx_spmv(ctx, A, _t(x).to(tdt), y)
        torch.cuda.synchronize()
        yref = oracle.spmv_csr(rp, col, val_r, x_r)
        bound = oracle.spmv_absbound(rp, col, val_r, x_r)
        assert_spmv_close(y.double().cpu().numpy(), yref, bound, TOL[dtype])
    finally:
        spx.spx_matrix_destroy(A)


def test_fullsize_powerlaw_ell_is_rejected(spx, ctx):
    rp, col, val = _mat("powerlaw_2m")
    with pytest.raises(spx.SpxError) as ei:
        spx.spx_matrix_create(ctx, "ell", _t(rp), _t(col), _t(val))
    assert ei.value.status == spx.SPX_ERR_TOO_LARGE


SOLVES = [("cg", "poisson128"), ("bicgstab", "convdiff128"), ("cgs", "convdiff128"), ("gmres", "convdiff128")]


@pytest.mark.parametrize("solver,prob", SOLVES)
def test_fullsize_solves(spx, ctx, solver, prob):
    rp, col, val = _mat(prob)
    n = rp.shape[0] - 1
    xs = np.random.default_rng(3).uniform(-1, 1, n)  # the bench's x*
    b = oracle.spmv_csr(rp, col, val, xs)
    A = spx.spx_matrix_create(ctx, "csr", _t(rp), _t(col), _t(val), flags=spx.SPX_MIXED_SHADOW)
    try:
        infos = {}
        for prec in ("f64", "mixed"):
            x = torch.zeros(n, dtype=torch.float64, device=DEV)
            info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 20000, restart=30, precision=prec)
            assert info.status == spx.SPX_CONVERGED, (prec, info)
            xh = x.cpu().numpy()
            rel = np.linalg.norm(b - oracle.spmv_csr(rp, col, val, xh)) / np.linalg.norm(b)
            assert rel <= residual_limit(rp, col, val, b, xh, 1e-10), (prec, rel)
            infos[prec] = info
        # the oracle's iteration count at full size (GMRES(30): MGS in the oracle,
        # classical Gram-Schmidt with reorthogonalisation on the GPU, same +-10% rule
        # as the small cases)
        kw = {"m": 30} if solver == "gmres" else {}
        _, oi = getattr(oracle, solver)(rp, col, val, b, tol=1e-10, maxit=20000, **kw)
        assert oi.status == oracle.CONVERGED
        slack = max(4, oi.iterations // (5 if solver == "cgs" else 10))
        assert abs(infos["f64"].iterations - oi.iterations) <= slack, (infos["f64"], oi)
    finally:
        spx.spx_matrix_destroy(A)


def test_fullsize_batch_sample(spx, ctx):
    nsys = 4096
    ro, no, rp, col, val = synth.batch_ragged_laplace(nsys, 100, 10000, seed=4)
    xs = np.random.default_rng(5).uniform(-1, 1, int(ro[-1]))
    sizes = np.diff(ro)
    rng = np.random.default_rng(12)
    sample = sorted(set(rng.choice(nsys, 20, replace=False).tolist() + [int(np.argmin(sizes)), int(np.argmax(sizes)),
                                                                         0, nsys - 1]))

    def system(s):
        r0, r1 = int(ro[s]), int(ro[s + 1])
        return rp[r0 + s: r1 + s + 1], col[no[s]: no[s + 1]], val[no[s]: no[s + 1]]

    b = np.empty_like(xs)
    for s in range(nsys):
        r0, r1 = int(ro[s]), int(ro[s + 1])
        lrp, lcol, lval = system(s)
        b[r0:r1] = oracle.spmv_csr(lrp, lcol, lval, xs[r0:r1])
    B = spx.spx_batch_create(ctx, ro, no, _t(rp), _t(col), _t(val), flags=spx.SPX_MIXED_SHADOW)
    try:
        for prec in ("f64", "mixed"):
            x = torch.zeros(int(ro[-1]), dtype=torch.float64, device=DEV)
            infos = spx.spx_batch_solve(ctx, B, _t(b), x, nsys, "cg", 1e-10, 20000, precision=prec)
            assert all(i.status == spx.SPX_CONVERGED for i in infos)
            xh = x.cpu().numpy()
            for s in sample:
                r0, r1 = int(ro[s]), int(ro[s + 1])
                lrp, lcol, lval = system(s)
                rel = np.linalg.norm(b[r0:r1] - oracle.spmv_csr(lrp, lcol, lval, xh[r0:r1])) / np.linalg.norm(b[r0:r1])
                assert rel <= residual_limit(lrp, lcol, lval, b[r0:r1], xh[r0:r1], 1e-10), (prec, s, rel)
                assert np.linalg.norm(xh[r0:r1] - xs[r0:r1]) / np.linalg.norm(xs[r0:r1]) <= 1e-6, (prec, s)
                if prec == "f64":
                    _, oi = oracle.cg(lrp, lcol, lval, b[r0:r1], tol=1e-10, maxit=20000)
                    assert abs(infos[s].iterations - oi.iterations) <= max(3, oi.iterations // 10), (s, infos[s], oi)
    finally:
        spx.spx_batch_destroy(B)
