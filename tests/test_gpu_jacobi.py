"""GPU Jacobi-preconditioned solves (M = diag A) against the CPU oracle:
true residual re-formed by the oracle's SpMV, iteration counts close to the
oracle's preconditioned methods, the column-scaling invariance of right
preconditioning reproduced on the GPU, one step on a diagonal matrix, and a
zero diagonal entry (taken as 1)."""
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


def _scale(rp, col, val, rs, cs):
    rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))
    return rp, col, val * rs[rows] * cs[col]


def _make(spx, ctx, fmt, rp, col, val, flags=0):
    return spx.spx_matrix_create(ctx, fmt, _t(rp), _t(col), _t(val), flags=flags)


def _relres(rp, col, val, b, x):
    return np.linalg.norm(b - oracle.spmv_csr(rp, col, val, x)) / np.linalg.norm(b)


def _problem(solver):
    rng = np.random.default_rng(21)
    if solver == "cg":  # SPD, symmetrically badly scaled
        rp, col, val = synth.laplace3d_7pt(12)
        s = np.exp(rng.uniform(-2.0, 2.0, size=rp.shape[0] - 1))
        rp, col, val = _scale(rp, col, val, s, s)
    else:  # nonsymmetric, rows badly scaled
        rp, col, val = synth.convdiff3d_upwind(12, peclet=10.0)
        rp, col, val = _scale(rp, col, val, np.exp(rng.uniform(-3.0, 3.0, size=rp.shape[0] - 1)),
                              np.ones(rp.shape[0] - 1))
    n = rp.shape[0] - 1
    xs = synth.uniform_vector(n, seed=3)
    return rp, col, val, xs, oracle.spmv_csr(rp, col, val, xs)


def _oracle(solver, rp, col, val, b, **kw):
    if solver == "gmres":
        return oracle.gmres(rp, col, val, b, m=30, **kw)
    return getattr(oracle, solver)(rp, col, val, b, **kw)


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo", "hyb"])
@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_jacobi_solve_matches_oracle(spx, ctx, solver, fmt):
    rp, col, val, xs, b = _problem(solver)
    A = _make(spx, ctx, fmt, rp, col, val)
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 20000, restart=30, precond="jacobi")
        _, oinfo = _oracle(solver, rp, col, val, b, tol=1e-10, maxit=20000, precond="jacobi")
        assert info.status == spx.SPX_CONVERGED, info
        xh = x.cpu().numpy()
        assert info.relres_true <= 1e-10 and _relres(rp, col, val, b, xh) <= residual_limit(rp, col, val, b, xh, 1e-10)
        slack = max(4, oinfo.iterations // (5 if solver == "cgs" else 10))
        assert abs(info.iterations - oinfo.iterations) <= slack, (info, oinfo)
        # the preconditioner pays off on these badly scaled matrices
        _, plain = _oracle(solver, rp, col, val, b, tol=1e-10, maxit=20000)
        assert plain.status != oracle.CONVERGED or plain.iterations > info.iterations
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["bicgstab", "cgs", "gmres"])
def test_right_jacobi_column_scaling_invariance_on_gpu(spx, ctx, solver):
    rp, col, val = synth.convdiff3d_upwind(10, peclet=10.0)
    n = rp.shape[0] - 1
    rng = np.random.default_rng(13)
    s = np.exp(rng.uniform(-2.0, 2.0, size=n))
    b = rng.standard_normal(n)
    xs = []
    for cs in (np.ones(n), s):
        rpc, colc, valc = _scale(rp, col, val, np.ones(n), cs)
        A = _make(spx, ctx, "csr", rpc, colc, valc)
        try:
            x = torch.zeros(n, dtype=torch.float64, device=DEV)
            spx.spx_solve_fixed(ctx, A, _t(b), x, solver, 6, restart=30, precond="jacobi")
            xs.append(x.cpu().numpy())
        finally:
            spx.spx_matrix_destroy(A)
    assert np.linalg.norm(s * xs[1] - xs[0]) <= 1e-8 * np.linalg.norm(xs[0])


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_jacobi_diagonal_matrix_one_step(spx, ctx, solver):
    n = 500
    d = np.random.default_rng(2).uniform(0.5, 20.0, size=n)
    rp, col = np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32)
    b = synth.uniform_vector(n, seed=4)
    A = _make(spx, ctx, "csr", rp, col, d)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-12, 100, restart=10, precond="jacobi")
        assert info.status == spx.SPX_CONVERGED and info.iterations == 1
        assert np.allclose(x.cpu().numpy(), b / d, rtol=1e-14, atol=0)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_jacobi_mixed_precision(spx, ctx, solver):
    rp, col, val, xs, b = _problem(solver)
    A = _make(spx, ctx, "csr", rp, col, val, flags=spx.SPX_MIXED_SHADOW)
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 20000, restart=30, precision="mixed",
                             precond="jacobi")
        assert info.status == spx.SPX_CONVERGED, info
        assert _relres(rp, col, val, b, x.cpu().numpy()) <= residual_limit(rp, col, val, b, x.cpu().numpy(), 1e-10)
    finally:
        spx.spx_matrix_destroy(A)


def test_zero_diagonal_entry_counts_as_one(spx, ctx):
    # identity with rows 0 and 1 swapped into a 2x2 [[0, 1], [1, 0]] block: diag(0, 0, 1, ...)
    n = 64
    dense = np.eye(n) * 3.0
    dense[0, 0] = dense[1, 1] = 0.0
    dense[0, 1] = dense[1, 0] = 1.0
    rp = np.zeros(n + 1, np.int32)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(dense[i])[0]
        cols.extend(nz)
        vals.extend(dense[i, nz])
        rp[i + 1] = len(cols)
    col, val = np.array(cols, np.int32), np.array(vals)
    b = synth.uniform_vector(n, seed=5)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, "gmres", 1e-12, 100, restart=10, precond="jacobi")
        assert info.status == spx.SPX_CONVERGED
        assert np.allclose(x.cpu().numpy(), np.linalg.solve(dense, b), rtol=0, atol=1e-11)
        _, oinfo = oracle.gmres(rp, col, val, b, m=10, tol=1e-12, maxit=100, precond="jacobi")
        assert oinfo.status == oracle.CONVERGED and info.iterations == oinfo.iterations
    finally:
        spx.spx_matrix_destroy(A)
