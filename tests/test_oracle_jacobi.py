"""Pins for the oracle's Jacobi-preconditioned solvers (M = diag(A); CPU only).

Facts used (none comes from the oracle): with M = diag(A), M^{-1} A = I for a
diagonal A, so every preconditioned method converges in one step; Jacobi-PCG
runs on D^{-1/2} A D^{-1/2}, which a symmetric diagonal scaling A -> S A S
leaves unchanged, so its iterates on S A S (right-hand side S b) are S^{-1}
times those on A; right preconditioning runs on A M^{-1}, which a column
scaling A -> A S leaves unchanged, so its iterates on A S are S^{-1} times
those on A with the same residuals.  The unpreconditioned methods break both
invariances, which shows that the pins test the preconditioner.
"""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import csr_from_dense, to_dense


def _diag(vals):
    n = len(vals)
    return np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(vals, dtype=np.float64)


def _scale(rp, col, val, rs, cs):
    """CSR of diag(rs) A diag(cs)."""
    rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))
    return rp, col, val * rs[rows] * cs[col]


def _run(solver, rp, col, val, b, j, precond):
    if solver == "gmres":
        return oracle.gmres(rp, col, val, b, m=40, tol=0.0, maxit=j, precond=precond)
    return getattr(oracle, solver)(rp, col, val, b, tol=0.0, maxit=j, precond=precond)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_jacobi_on_diagonal_matrix_is_one_step(solver):
    d = np.random.default_rng(2).uniform(0.5, 20.0, size=25)
    rp, col, val = _diag(d)
    b = np.random.default_rng(3).standard_normal(25)
    if solver == "gmres":
        x, info = oracle.gmres(rp, col, val, b, m=10, tol=1e-12, precond="jacobi")
    else:
        x, info = getattr(oracle, solver)(rp, col, val, b, tol=1e-12, precond="jacobi")
    assert info.status == oracle.CONVERGED and info.iterations == 1
    assert np.allclose(x, b / d, rtol=1e-14, atol=0)


@pytest.mark.parametrize("j", [2, 5, 9])
def test_pcg_jacobi_invariant_under_symmetric_scaling(j):
    rp, col, val = synth.laplace2d_5pt(12)
    n = rp.shape[0] - 1
    rng = np.random.default_rng(11)
    s = np.exp(rng.uniform(-2.0, 2.0, size=n))
    b = rng.standard_normal(n)
    rps, cols, vals = _scale(rp, col, val, s, s)
    x, _ = _run("cg", rp, col, val, b, j, "jacobi")
    xs, _ = _run("cg", rps, cols, vals, s * b, j, "jacobi")
    assert np.linalg.norm(s * xs - x) <= 1e-10 * np.linalg.norm(x)
    # plain CG is not invariant: the pin is about the preconditioner
    x0, _ = _run("cg", rp, col, val, b, j, None)
    xs0, _ = _run("cg", rps, cols, vals, s * b, j, None)
    assert np.linalg.norm(s * xs0 - x0) > 1e-3 * np.linalg.norm(x0)


@pytest.mark.parametrize("solver", ["bicgstab", "cgs", "gmres"])
@pytest.mark.parametrize("j", [2, 6])
def test_right_jacobi_invariant_under_column_scaling(solver, j):
    m = 6
    rp, col, val = synth.convdiff3d_upwind(m, peclet=10.0)
    n = m**3
    rng = np.random.default_rng(13)
    s = np.exp(rng.uniform(-2.0, 2.0, size=n))
    b = rng.standard_normal(n)
    rpc, colc, valc = _scale(rp, col, val, np.ones(n), s)
    x, info = _run(solver, rp, col, val, b, j, "jacobi")
    xc, infoc = _run(solver, rpc, colc, valc, b, j, "jacobi")
    assert np.linalg.norm(s * xc - x) <= 1e-9 * np.linalg.norm(x)
    assert infoc.relres_true == pytest.approx(info.relres_true, rel=1e-9)
    x0, _ = _run(solver, rp, col, val, b, j, None)
    xc0, _ = _run(solver, rpc, colc, valc, b, j, None)
    assert np.linalg.norm(s * xc0 - x0) > 1e-3 * np.linalg.norm(x0)


@pytest.mark.parametrize("solver", ["bicgstab", "cgs", "gmres"])
def test_jacobi_solves_badly_row_scaled_convdiff(solver):
    m = 8
    rp, col, val = synth.convdiff3d_upwind(m, peclet=10.0)
    n = m**3
    rs = np.exp(np.random.default_rng(5).uniform(-3.0, 3.0, size=n))
    rp, col, val = _scale(rp, col, val, rs, np.ones(n))
    xs = synth.uniform_vector(n, seed=3)
    b = oracle.spmv_csr(rp, col, val, xs)
    kw = {"m": 30} if solver == "gmres" else {}
    x, info = getattr(oracle, solver)(rp, col, val, b, tol=1e-10, maxit=3000, precond="jacobi", **kw)
    assert info.status == oracle.CONVERGED and info.relres_true <= 1e-10
    ref = np.linalg.solve(to_dense(rp, col, val), b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-7
    _, plain = getattr(oracle, solver)(rp, col, val, b, tol=1e-10, maxit=3000, **kw)
    assert plain.status != oracle.CONVERGED or plain.iterations > info.iterations


def test_planted_mistake_in_preconditioned_update_is_caught():
    m = 6
    rp, col, val = synth.convdiff3d_upwind(m, peclet=10.0)
    n = m**3
    rng = np.random.default_rng(13)
    s = np.exp(rng.uniform(-2.0, 2.0, size=n))
    b = rng.standard_normal(n)
    rpc, colc, valc = _scale(rp, col, val, np.ones(n), s)
    x, _ = oracle.bicgstab(rp, col, val, b, tol=0.0, maxit=4, precond="jacobi", mutant=7)
    xc, _ = oracle.bicgstab(rpc, colc, valc, b, tol=0.0, maxit=4, precond="jacobi", mutant=7)
    assert np.linalg.norm(s * xc - x) > 1e-6 * np.linalg.norm(x)
