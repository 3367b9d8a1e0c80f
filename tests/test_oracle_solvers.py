"""Pins for the oracle's Krylov solvers (CPU only).

Facts used (none comes from the oracle itself): CG terminates in at most n
steps on SPD systems and in at most d steps when b lies in a d-dimensional
invariant subspace with d distinct eigenvalues; CG on an eigenvector converges
in one step to v / lambda; BiCGSTAB and CGS on c*I converge in one step; CGS's
residual polynomial is the square of CG's on an SPD matrix with r^ = r0 (by
its construction), so it also terminates in d steps; GMRES on a matrix whose
minimal polynomial has degree d terminates in at most d steps and its residual
never increases; manufactured solutions b = A x* with the error bounded by
kappa * tol; numpy's dense LU as an independent solve; the rounding bounds of
FP32 and FP64 arithmetic (unit roundoffs 2^-24 and 2^-53) for each cycle of
iterative refinement on c*I.
"""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import csr_from_dense, laplace1d, to_dense


def _spd(rng, n, kappa):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, kappa, n)
    return (q * ev) @ q.T, q, ev


# ---------------------------------------------------------------- CG
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n", [2, 5, 8])
def test_cg_terminates_within_n_steps(seed, n):
    rng = np.random.default_rng(seed)
    a, _, _ = _spd(rng, n, 100.0)
    rp, col, val = csr_from_dense(a)
    b = rng.standard_normal(n)
    # exact arithmetic terminates in n steps; in double the n-th residual is at
    # the level of kappa * eps * (growth), far below what a wrong term leaves.
    x, info = oracle.cg(rp, col, val, b, tol=1e-8, maxit=n)
    assert info.status == oracle.CONVERGED
    assert info.iterations <= n
    assert info.relres_true <= 1e-8
    x, info = oracle.cg(rp, col, val, b, tol=1e-10, maxit=n + 3)
    assert info.status == oracle.CONVERGED and info.relres_true <= 1e-10
    assert np.allclose(x, np.linalg.solve(a, b), rtol=0, atol=1e-8 * np.abs(np.linalg.solve(a, b)).max())


def test_cg_on_eigenvector_converges_in_one_step():
    m = 9
    rp, col, val = laplace1d(m)
    i = np.arange(1, m + 1)
    v = np.sin(i * 2 * np.pi / (m + 1))
    lam = 2 - 2 * np.cos(2 * np.pi / (m + 1))
    x, info = oracle.cg(rp, col, val, v, tol=1e-12)
    assert info.iterations == 1
    assert np.allclose(x, v / lam, rtol=0, atol=1e-13)


def test_cg_terminates_in_d_steps_for_d_eigencomponents():
    rng = np.random.default_rng(5)
    n = 12
    a, q, ev = _spd(rng, n, 50.0)
    rp, col, val = csr_from_dense(a)
    for d in (1, 2, 3, 4):
        b = q[:, :d] @ rng.uniform(1, 2, size=d)
        _, info = oracle.cg(rp, col, val, b, tol=1e-10, maxit=50)
        assert info.status == oracle.CONVERGED
        assert info.iterations <= d


def test_cg_manufactured_laplace2d():
    rp, col, val = synth.laplace2d_5pt(24)
    n = 24 * 24
    xs = synth.uniform_vector(n, seed=0)
    b = oracle.spmv_csr(rp, col, val, xs)
    x, info = oracle.cg(rp, col, val, b, tol=1e-10, maxit=2000)
    kappa = (4 + 4 * np.cos(np.pi / 25)) / (4 - 4 * np.cos(np.pi / 25))
    assert info.status == oracle.CONVERGED and info.relres_true <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-10


def test_cg_zero_rhs_and_max_iter():
    rp, col, val = synth.laplace2d_5pt(8)
    x, info = oracle.cg(rp, col, val, np.zeros(64))
    assert info.iterations == 0 and np.all(x == 0) and info.status == oracle.CONVERGED
    _, info = oracle.cg(rp, col, val, np.ones(64), tol=1e-14, maxit=3)
    assert info.status == oracle.MAX_ITER and info.iterations == 3


def test_cg_history_is_recorded():
    rp, col, val = synth.laplace2d_5pt(10)
    b = np.ones(100)
    _, info, h = oracle.cg(rp, col, val, b, tol=1e-10, hist=True)
    assert h.shape[0] == info.iterations + 1
    assert h[0] == pytest.approx(1.0) and h[-1] <= 1e-10


def test_cg_planted_sign_mistake_is_caught():
    rng = np.random.default_rng(0)
    a, _, _ = _spd(rng, 8, 100.0)
    rp, col, val = csr_from_dense(a)
    _, info = oracle.cg(rp, col, val, rng.standard_normal(8), tol=1e-10, maxit=8, mutant=3)
    assert not (info.status == oracle.CONVERGED and info.iterations <= 8)


# ---------------------------------------------------------------- BiCGSTAB
@pytest.mark.parametrize("c", [1.0, 3.5, -2.0])
def test_bicgstab_scaled_identity_one_step(c):
    n = 17
    rp = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    val = np.full(n, c)
    b = np.random.default_rng(1).standard_normal(n)
    x, info = oracle.bicgstab(rp, col, val, b, tol=1e-12)
    assert info.iterations == 1 and info.status == oracle.CONVERGED
    assert np.allclose(x, b / c, rtol=1e-15, atol=0)


def test_bicgstab_convdiff_manufactured():
    m = 8
    rp, col, val = synth.convdiff3d_upwind(m, peclet=10.0)
    n = m**3
    xs = synth.uniform_vector(n, seed=3)
    b = oracle.spmv_csr(rp, col, val, xs)
    x, info = oracle.bicgstab(rp, col, val, b, tol=1e-10, maxit=1000)
    assert info.status == oracle.CONVERGED and info.relres_true <= 1e-10
    ref = np.linalg.solve(to_dense(rp, col, val), b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-8


def test_bicgstab_planted_mistake_is_caught():
    m = 6
    rp, col, val = synth.convdiff3d_upwind(m)
    b = oracle.spmv_csr(rp, col, val, synth.uniform_vector(m**3, seed=3))
    _, good = oracle.bicgstab(rp, col, val, b, tol=1e-10, maxit=400)
    _, bad = oracle.bicgstab(rp, col, val, b, tol=1e-10, maxit=400, mutant=4)
    assert good.status == oracle.CONVERGED
    assert bad.status != oracle.CONVERGED or bad.relres_true > 1e-10


# ---------------------------------------------------------------- CGS
def _diag(vals):
    n = len(vals)
    return np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(vals, dtype=np.float64)


@pytest.mark.parametrize("c", [1.0, 3.5, -2.0])
def test_cgs_scaled_identity_one_step(c):
    rp, col, val = _diag(np.full(17, c))
    b = np.random.default_rng(1).standard_normal(17)
    x, info = oracle.cgs(rp, col, val, b, tol=1e-12)
    assert info.iterations == 1 and info.status == oracle.CONVERGED
    assert np.allclose(x, b / c, rtol=1e-15, atol=0)


@pytest.mark.parametrize("j", [1, 2, 3, 4])
def test_cgs_residual_is_cg_residual_polynomial_squared(j):
    # A = diag(lam), r^ = r0 = b: CG's residual is phi_j(A) b, CGS's is
    # phi_j(A)^2 b, so componentwise r_cgs[i] * b[i] = r_cg[i]^2.
    rng = np.random.default_rng(7)
    lam = rng.uniform(1.0, 10.0, size=30)
    rp, col, val = _diag(lam)
    b = rng.uniform(0.5, 1.5, size=30) * rng.choice([-1.0, 1.0], size=30)
    x_cg, _ = oracle.cg(rp, col, val, b, tol=0.0, maxit=j)
    x_cgs, info = oracle.cgs(rp, col, val, b, tol=0.0, maxit=j)
    assert info.iterations == j
    r_cg = b - lam * x_cg
    r_cgs = b - lam * x_cgs
    scale = np.abs(b).max() ** 2
    assert np.max(np.abs(r_cgs * b - r_cg**2)) <= 1e-12 * scale
    assert np.linalg.norm(r_cgs) > 1e-8  # not converged yet: the identity is not trivially 0 = 0


@pytest.mark.parametrize("d", [2, 3, 5])
def test_cgs_terminates_in_d_steps_for_d_distinct_eigenvalues(d):
    rng = np.random.default_rng(d)
    ev = np.linspace(1.0, 4.0, d)
    lam = ev[rng.integers(0, d, size=40)]
    lam[:d] = ev  # every eigenvalue present
    rp, col, val = _diag(lam)
    b = rng.uniform(0.5, 1.5, size=40)
    _, info = oracle.cgs(rp, col, val, b, tol=1e-10, maxit=d)
    assert info.status == oracle.CONVERGED and info.iterations <= d
    _, short = oracle.cgs(rp, col, val, b, tol=0.0, maxit=d - 1)
    assert short.relres_true > 1e-6  # a degree d-1 polynomial cannot vanish on d eigenvalues


def test_cgs_convdiff_manufactured():
    m = 8
    rp, col, val = synth.convdiff3d_upwind(m, peclet=10.0)
    n = m**3
    xs = synth.uniform_vector(n, seed=3)
    b = oracle.spmv_csr(rp, col, val, xs)
    x, info = oracle.cgs(rp, col, val, b, tol=1e-10, maxit=1000)
    assert info.status == oracle.CONVERGED and info.relres_true <= 1e-10
    ref = np.linalg.solve(to_dense(rp, col, val), b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-8


def test_cgs_planted_mistake_is_caught():
    rng = np.random.default_rng(7)
    lam = rng.uniform(1.0, 10.0, size=30)
    rp, col, val = _diag(lam)
    b = rng.uniform(0.5, 1.5, size=30)
    x_cg, _ = oracle.cg(rp, col, val, b, tol=0.0, maxit=2)
    x_bad, _ = oracle.cgs(rp, col, val, b, tol=0.0, maxit=2, mutant=6)
    r_cg, r_bad = b - lam * x_cg, b - lam * x_bad
    assert np.max(np.abs(r_bad * b - r_cg**2)) > 1e-6


# ---------------------------------------------------------------- GMRES
@pytest.mark.parametrize("d", [1, 2, 4, 7])
def test_gmres_terminates_at_minimal_polynomial_degree(d):
    # Diagonal matrix with d distinct values (repeated): minimal polynomial degree d.
    n = 40
    vals = np.linspace(1.0, 5.0, d)
    diag = vals[np.arange(n) % d]
    rp = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    b = np.random.default_rng(d).standard_normal(n)
    x, info = oracle.gmres(rp, col, diag, b, m=30, tol=1e-11)
    assert info.status == oracle.CONVERGED and info.iterations <= d
    assert np.allclose(x, b / diag, rtol=1e-10, atol=0)


@pytest.mark.parametrize("m", [3, 10, 30])
def test_gmres_residual_monotone(m):
    k = 6
    rp, col, val = synth.convdiff3d_upwind(k)
    b = np.ones(k**3)
    _, info, h = oracle.gmres(rp, col, val, b, m=m, tol=1e-10, maxit=3000, hist=True)
    assert info.status == oracle.CONVERGED
    assert np.all(np.diff(h) <= 1e-13)


def test_gmres_full_when_m_at_least_n():
    rng = np.random.default_rng(9)
    n = 12
    a = rng.standard_normal((n, n)) + 4 * np.eye(n)
    rp, col, val = csr_from_dense(a)
    b = rng.standard_normal(n)
    x, info = oracle.gmres(rp, col, val, b, m=n, tol=1e-10)
    assert info.iterations <= n and info.status == oracle.CONVERGED
    assert np.allclose(x, np.linalg.solve(a, b), rtol=0, atol=1e-8)


def test_gmres_matches_cg_final_residual_on_spd():
    rp, col, val = synth.laplace2d_5pt(16)
    b = oracle.spmv_csr(rp, col, val, synth.uniform_vector(256, 0))
    _, icg = oracle.cg(rp, col, val, b, tol=1e-10)
    _, igm = oracle.gmres(rp, col, val, b, m=300, tol=1e-10)
    assert icg.relres_true <= 1e-10 and igm.relres_true <= 1e-10
    # full GMRES minimises the residual over the Krylov space: never more steps than CG
    assert igm.iterations <= icg.iterations


def test_gmres_planted_mistake_is_caught():
    rng = np.random.default_rng(9)
    n = 12
    a = rng.standard_normal((n, n)) + 4 * np.eye(n)
    rp, col, val = csr_from_dense(a)
    b = rng.standard_normal(n)
    x, info = oracle.gmres(rp, col, val, b, m=n, tol=1e-10, maxit=40, mutant=5)
    assert not np.allclose(x, np.linalg.solve(a, b), rtol=0, atol=1e-8) or info.relres_true > 1e-10


# ---------------------------------------------------------------- IR
def test_ir_reaches_fp64_tolerance_cg():
    rp, col, val = synth.laplace3d_7pt(10)
    xs = synth.uniform_vector(1000, 3)
    b = oracle.spmv_csr(rp, col, val, xs)
    x, info = oracle.ir(rp, col, val, b, solver="cg", tol=1e-10)
    assert info.status == oracle.CONVERGED and info.relres_true <= 1e-10
    assert info.restarts >= 2  # an FP32 inner solve alone cannot reach 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-9


def test_ir_reaches_fp64_tolerance_bicgstab():
    rp, col, val = synth.convdiff3d_upwind(8)
    xs = synth.uniform_vector(512, 3)
    b = oracle.spmv_csr(rp, col, val, xs)
    x, info = oracle.ir(rp, col, val, b, solver="bicgstab", tol=1e-10)
    assert info.status == oracle.CONVERGED and info.relres_true <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-8


def test_ir_reaches_fp64_tolerance_cgs():
    rp, col, val = synth.convdiff3d_upwind(8)
    xs = synth.uniform_vector(512, 3)
    b = oracle.spmv_csr(rp, col, val, xs)
    x, info = oracle.ir(rp, col, val, b, solver="cgs", tol=1e-10)
    assert info.status == oracle.CONVERGED and info.relres_true <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-8


def test_ir_cgs_stall_rule_ends_blown_up_cycles():
    """FP32 CGS inside refinement on the 64^3 upwind convection-diffusion
    matrix: after the first cycle the inner residual blows up (CGS squares its
    residual polynomial); with the 500-iteration cap alone the solve needs
    711 inner iterations, with the 20-iteration stall rule far fewer.  The
    true residual is recomputed here with scipy, independently of the oracle."""
    import scipy.sparse as sp
    rp, col, val = synth.convdiff3d_upwind(64)
    n = rp.shape[0] - 1
    xs = np.random.default_rng(3).uniform(-1, 1, n)
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    b = A @ xs
    x, info = oracle.ir(rp, col, val, b, solver="cgs", tol=1e-10)
    assert info.status == oracle.CONVERGED
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-10
    assert info.restarts >= 3  # more than one blown-up cycle was cut short and restarted
    assert info.iterations < 300, info


# ---------------------------------------------------------------- IR: the iterate path
# On A = c*I with c a power of two every FP32 inner solver takes one step and
# returns d = r32 / c exactly (see the one-step pins above), so a refinement
# cycle adds to x the FP32 rounding of the normalised FP64 residual, scaled back.
# Rounding arithmetic then fixes each cycle's result: after one cycle
# |b_i - c x_i| <= 2^-24 |b_i| (one FP32 rounding, plus FP64 roundings of
# order 2^-53); after two, <= 2^-47 |b_i| (the second cycle rounds a residual
# already 2^-24 small, and the FP64 update adds at most 2^-53 |b_i|).  So a solve
# to 1e-10 ends after exactly two cycles.  A residual or an update taken in FP32,
# a correction not scaled back by the residual norm, or a wrong sign breaks one
# of these bounds.
def _scaled_identity(n, c):
    return np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, c)


def _ir_scaled_identity_pins(solver, c, mutant=0):
    """The cycle-by-cycle facts above, each as a bool."""
    n = 257
    rp, col, val = _scaled_identity(n, c)
    b = np.random.default_rng(5).uniform(-1, 1, n)
    b[np.abs(b) < 1e-3] = 0.5  # keep every component well inside the normal FP32 range after scaling
    x1, i1 = oracle.ir(rp, col, val, b, solver=solver, tol=1e-10, max_outer=1, mutant=mutant)
    err1 = np.abs(b - c * x1)
    x2, _ = oracle.ir(rp, col, val, b, solver=solver, tol=1e-10, max_outer=2, mutant=mutant)
    err2 = np.abs(b - c * x2)
    x, info = oracle.ir(rp, col, val, b, solver=solver, tol=1e-10, mutant=mutant)
    return {
        "one cycle stops": i1.status == oracle.MAX_ITER and i1.restarts == 1,
        "one cycle: 2^-24": bool(np.all(err1 <= 2.0 ** -24 * (1 + 1e-6) * np.abs(b))),
        "one cycle leaves an FP32 rounding": bool(np.max(err1 / np.abs(b)) > 2.0 ** -30),
        "two cycles: 2^-47": bool(np.all(err2 <= 2.0 ** -47 * np.abs(b))),
        "converged after two cycles": info.status == oracle.CONVERGED and info.restarts == 2,
        "one inner step per cycle": info.iterations == 2,
        "same two cycles": bool(np.array_equal(x, x2)),
    }


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs"])
@pytest.mark.parametrize("c", [0.25, 8.0])
def test_ir_cycles_on_scaled_identity_follow_fp32_rounding(solver, c):
    pins = _ir_scaled_identity_pins(solver, c)
    assert all(pins.values()), pins


@pytest.mark.parametrize("mutant", [9, 10])
def test_ir_planted_update_mistakes_are_caught(mutant):
    """9: the correction is not scaled back by the residual norm; 10: the update is
    rounded to FP32.  Each breaks a cycle-by-cycle pin."""
    pins = _ir_scaled_identity_pins("cg", 0.25, mutant=mutant)
    assert not all(pins.values()), pins


def test_ir_planted_fp32_residual_is_caught():
    """11: the outer residual uses the FP32 values.  On c*I with c a power of two
    that changes nothing, so the pin is a matrix whose values FP32 cannot hold:
    refinement then converges to the FP32 matrix's solution, and the true FP64
    residual, recomputed with scipy, stays far above the tolerance."""
    import scipy.sparse as sp
    rp, col, val = synth.convdiff3d_upwind(8)
    n = rp.shape[0] - 1
    assert np.any(val.astype(np.float32).astype(np.float64) != val)
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    b = A @ np.random.default_rng(3).uniform(-1, 1, n)
    for mutant, ok in ((0, True), (11, False)):
        x, _ = oracle.ir(rp, col, val, b, solver="bicgstab", tol=1e-10, mutant=mutant)
        assert (np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-10) == ok, mutant
