"""The one-launch solve on a thread-block cluster (SPX_SOLVE_ONE_CLUSTER)
against the CPU oracle: CG, BiCGSTAB and CGS in FP64, FP32 and mixed
precision, on systems whose rows split unevenly over the cluster's blocks
(8-block clusters below 65 536 rows, 16-block clusters above), with tiny
systems where some blocks own no row, b = 0, the iteration limit, bitwise
repeatability and the combinations the route refuses."""
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


_CACHE = {}


def _problem(name):
    if name in _CACHE:
        return _CACHE[name]
    if name == "lap3d_20":          # 8000 rows: blocks of 1024 rows, the last one 832
        rp, col, val = synth.laplace3d_7pt(20)
    elif name == "lap3d_41":        # 68 921 rows: 16 blocks of 4320 rows, the last one 4121
        rp, col, val = synth.laplace3d_7pt(41)
    elif name == "convdiff_16":     # 4096 rows, nonsymmetric
        rp, col, val = synth.convdiff3d_upwind(16)
    elif name == "diagdom_70001":   # random columns over the whole matrix, 8..32 entries per row
        rp, col, val = synth.DiagDomFamily(70001, seed=11).matrix(70001)
    elif name == "lap1d_5":         # 5 rows: 7 of 8 blocks own none
        rp, col, val = _lap1d(5)
    else:
        raise KeyError(name)
    n = rp.shape[0] - 1
    xs = synth.uniform_vector(n, seed=3)
    b = oracle.spmv_csr(rp, col, val, xs)
    _CACHE[name] = (rp, col, val, xs, b)
    return _CACHE[name]


def _lap1d(n):
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
                vals.append(v)
    rp = np.zeros(n + 1, np.int32)
    np.add.at(rp, np.array(rows) + 1, 1)
    return np.cumsum(rp).astype(np.int32), np.array(cols, np.int32), np.array(vals)


def _true_relres(rp, col, val, b, x):
    return np.linalg.norm(b - oracle.spmv_csr(rp, col, val, x)) / np.linalg.norm(b)


ORACLE = {"cg": oracle.cg, "bicgstab": oracle.bicgstab, "cgs": oracle.cgs}


def _solve(spx, ctx, prob, solver, precision, tol, maxit=20000):
    rp, col, val, xs, b = _problem(prob)
    f32 = precision == "f32"
    A = spx.spx_matrix_create(ctx, "csr", _t(rp), _t(col), _t(val).float() if f32 else _t(val),
                              flags=spx.SPX_MIXED_SHADOW if precision == "mixed" else 0)
    try:
        bt = _t(b).float() if f32 else _t(b)
        x = torch.zeros_like(bt)
        info = spx.spx_solve(ctx, A, bt, x, solver, tol, maxit, precision=precision, one_cluster=True)
        x2 = torch.zeros_like(bt)
        info2 = spx.spx_solve(ctx, A, bt, x2, solver, tol, maxit, precision=precision, one_cluster=True)
        assert torch.equal(x, x2) and info2.iterations == info.iterations  # no dependence on timing
        return info, x.double().cpu().numpy()
    finally:
        spx.spx_matrix_destroy(A)


# CG on the symmetric matrices; BiCGSTAB and CGS on all of them
CASES = [(s, p) for p in ("lap3d_20", "lap3d_41", "convdiff_16", "diagdom_70001") for s in ("cg", "bicgstab", "cgs")
         if s != "cg" or p.startswith("lap")]


@pytest.mark.parametrize("solver,prob", CASES)
def test_fp64_against_oracle(spx, ctx, prob, solver):
    rp, col, val, xs, b = _problem(prob)
    info, xh = _solve(spx, ctx, prob, solver, "f64", 1e-10)
    assert info.status == spx.SPX_CONVERGED, info
    assert info.relres_true <= 1e-10
    assert _true_relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, 1e-10)
    assert np.linalg.norm(xh - xs) / np.linalg.norm(xs) <= 1e-7
    _, oi = ORACLE[solver](rp, col, val, b, tol=1e-10, maxit=20000)
    # BiCGSTAB / CGS convergence is irregular: rounding moves the stop by a few steps
    slack = max(3, oi.iterations // 10) if solver == "cg" else max(6, oi.iterations // 5)
    assert abs(info.iterations - oi.iterations) <= slack, (info, oi)


@pytest.mark.parametrize("solver,prob", CASES)
def test_mixed_against_oracle(spx, ctx, prob, solver):
    rp, col, val, xs, b = _problem(prob)
    info, xh = _solve(spx, ctx, prob, solver, "mixed", 1e-10)
    assert info.status == spx.SPX_CONVERGED, info
    assert info.relres_true <= 1e-10
    assert _true_relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, 1e-10)
    assert np.linalg.norm(xh - xs) / np.linalg.norm(xs) <= 1e-7
    assert info.inner_iterations == info.iterations > 0
    if solver == "cg":  # reliable updates, as spx_solve runs mixed CG
        _, oi = oracle.cg_reliable(rp, col, val, b, tol=1e-10)
        assert oi.status == oracle.CONVERGED
        assert abs(info.iterations - oi.iterations) <= max(3, oi.iterations // 10), (info, oi)
        assert abs(info.restarts - oi.restarts) <= 3, (info, oi)
    else:  # FP32 inner solves to 1e-4, cycle by cycle
        _, oi = oracle.ir(rp, col, val, b, solver=solver, tol=1e-10)
        assert oi.status == oracle.CONVERGED
        assert abs(info.restarts - oi.restarts) <= 2, (info, oi)


@pytest.mark.parametrize("prob", ["lap3d_20", "lap3d_41"])
@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs"])
def test_fp32(spx, ctx, prob, solver):
    rp, col, val, xs, b = _problem(prob)
    info, xh = _solve(spx, ctx, prob, solver, "f32", 1e-5)
    assert info.status == spx.SPX_CONVERGED, info
    v32 = val.astype(np.float32).astype(np.float64)
    b32 = b.astype(np.float32).astype(np.float64)
    assert _true_relres(rp, col, v32, b32, xh) <= 2e-5


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs"])
@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_tiny_system_most_blocks_idle(spx, ctx, solver, precision):
    rp, col, val, xs, b = _problem("lap1d_5")
    info, xh = _solve(spx, ctx, "lap1d_5", solver, precision, 1e-12)
    assert info.status == spx.SPX_CONVERGED, info
    xd = np.linalg.solve(_dense(rp, col, val), b)
    assert np.allclose(xh, xd, rtol=1e-10, atol=1e-12)


def _dense(rp, col, val):
    n = rp.shape[0] - 1
    D = np.zeros((n, n))
    for i in range(n):
        D[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    return D


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_zero_rhs_and_iteration_limit(spx, ctx, precision):
    rp, col, val, xs, b = _problem("lap3d_20")
    A = spx.spx_matrix_create(ctx, "csr", _t(rp), _t(col), _t(val),
                              flags=spx.SPX_MIXED_SHADOW if precision == "mixed" else 0)
    try:
        x = torch.ones(b.shape[0], dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, torch.zeros_like(x), x, "cg", 1e-10, 100, precision=precision,
                             one_cluster=True)
        assert info.status == spx.SPX_CONVERGED and not x.any()
        x = torch.zeros_like(x)
        info = spx.spx_solve(ctx, A, _t(b), x, "cg", 1e-10, 5, precision=precision, one_cluster=True)
        assert info.status == spx.SPX_MAX_ITER, info
        assert info.iterations == 5 if precision == "f64" else info.iterations >= 5
    finally:
        spx.spx_matrix_destroy(A)


def test_refused_combinations(spx, ctx):
    rp, col, val, xs, b = _problem("lap3d_20")
    A = spx.spx_matrix_create(ctx, "csr", _t(rp), _t(col), _t(val))
    E = spx.spx_matrix_create(ctx, "ell", _t(rp), _t(col), _t(val))
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        for kw in ({"solver": "gmres"}, {"solver": "cg", "precond": "jacobi"},
                   {"solver": "cg", "precision": "f32"}):
            with pytest.raises(spx.SpxError) as e:
                spx.spx_solve(ctx, A, _t(b), x, tol=1e-10, max_iter=100, one_cluster=True, **kw)
            assert e.value.status == spx.SPX_ERR_UNSUPPORTED
        with pytest.raises(spx.SpxError) as e:
            spx.spx_solve(ctx, E, _t(b), x, "cg", 1e-10, 100, one_cluster=True)
        assert e.value.status == spx.SPX_ERR_UNSUPPORTED
    finally:
        spx.spx_matrix_destroy(A)
        spx.spx_matrix_destroy(E)
