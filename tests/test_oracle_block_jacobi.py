"""Pins for the oracle's block-Jacobi preconditioner (CPU only).

M is the block diagonal of A with blocks of bs consecutive rows and columns.
Facts used (none comes from the oracle): the block inverses are what
numpy.linalg.inv gives for the dense diagonal blocks; bs = 1 is Jacobi; for a
block-diagonal A, M^{-1} A = I, so every preconditioned method converges in one
step to A^{-1} b; right preconditioning runs on A M^{-1}, which A -> A S leaves
unchanged for any nonsingular block-diagonal S with the same blocks (the block
diagonal of A S is D S), so the iterates on A S are S^{-1} times those on A;
block-PCG runs on the operator M^{-1} A, and A -> S^T A S with a block-diagonal
S maps it to S^{-1} M^{-1} A S, so its iterates on S^T A S (right-hand side
S^T b) are S^{-1} times those on A.  A transposed, shifted or mis-sized block
breaks these.
"""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import csr_from_dense, to_dense


def _blocks_dense(a, bs):
    n = a.shape[0]
    out = []
    for c0 in range(0, n, bs):
        blk = np.eye(bs)
        m = min(bs, n - c0)
        blk[:m, :m] = a[c0:c0 + m, c0:c0 + m]
        out.append(np.linalg.inv(blk))
    return np.array(out)


def _block_diag(blocks, n):
    bs = blocks.shape[1]
    s = np.zeros((n, n))
    for k, blk in enumerate(blocks):
        c0 = k * bs
        m = min(bs, n - c0)
        s[c0:c0 + m, c0:c0 + m] = blk[:m, :m]
    return s


@pytest.mark.parametrize("bs,n", [(1, 17), (2, 17), (4, 16), (4, 18), (8, 30), (32, 70)])
def test_block_inverse_matches_numpy(bs, n):
    rng = np.random.default_rng(bs * 100 + n)
    a = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.4)
    a += np.diag(rng.uniform(1.0, 3.0, n))
    rp, col, val = csr_from_dense(a)
    got = oracle.block_jacobi_inv(rp, col, val, bs)
    want = _blocks_dense(a, bs)
    assert got.shape == want.shape
    assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_block_inverse_needs_pivoting_and_sums_duplicates():
    # a nonsingular block with a zero leading diagonal entry, and an entry given twice
    a = np.array([[0.0, 2.0, 0.0, 0.0], [3.0, 1.0, 0.0, 5.0], [0.0, 0.0, 4.0, 1.0], [0.0, 7.0, 1.0, 2.0]])
    rp, col, val = csr_from_dense(a)
    # split a[2][3] = 1 into 0.25 + 0.75 stored twice
    k = int(np.nonzero((col[rp[2]:rp[3]] == 3))[0][0]) + rp[2]
    col = np.insert(col, k + 1, 3)
    val = np.insert(val, k + 1, 0.75)
    val[k] = 0.25
    rp = rp.copy()
    rp[3:] += 1
    got = oracle.block_jacobi_inv(rp, col, val, 2)
    assert np.allclose(got, _blocks_dense(a, 2), rtol=0, atol=1e-14)


def test_singular_block_is_identity_and_bs1_is_jacobi():
    a = np.diag([2.0, 4.0, 0.0, 5.0, 8.0, 1.0])
    a[2, 3] = 1.0  # block [2,3] = [[0,1],[0,5]] is singular
    rp, col, val = csr_from_dense(a)
    got = oracle.block_jacobi_inv(rp, col, val, 2)
    assert np.array_equal(got[1], np.eye(2))
    assert np.array_equal(got[0], np.diag([0.5, 0.25]))
    d1 = oracle.block_jacobi_inv(rp, col, val, 1)[:, 0, 0]
    diag = np.diag(a)
    assert np.array_equal(d1, np.where(diag != 0, 1.0 / np.where(diag != 0, diag, 1.0), 1.0))


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_bs1_block_jacobi_is_jacobi_bitwise(solver):
    rp, col, val = synth.convdiff3d_upwind(6) if solver != "cg" else synth.laplace3d_7pt(6)
    n = rp.shape[0] - 1
    b = np.random.default_rng(5).standard_normal(n)
    kw = {"m": 20} if solver == "gmres" else {}
    xj, ij = getattr(oracle, solver)(rp, col, val, b, tol=1e-10, precond="jacobi", **kw)
    xb, ib = getattr(oracle, solver)(rp, col, val, b, tol=1e-10, precond="block_jacobi", block_size=1, **kw)
    assert np.array_equal(xj, xb) and ij == ib


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
@pytest.mark.parametrize("bs", [2, 4, 8])
def test_block_diagonal_matrix_is_one_step(solver, bs):
    rng = np.random.default_rng(bs)
    n = 5 * bs + bs // 2  # a ragged last block
    a = np.zeros((n, n))
    for c0 in range(0, n, bs):
        m = min(bs, n - c0)
        g = rng.standard_normal((m, m))
        a[c0:c0 + m, c0:c0 + m] = g @ g.T + m * np.eye(m) if solver == "cg" else g + 2 * m * np.eye(m)
    rp, col, val = csr_from_dense(a)
    b = rng.standard_normal(n)
    kw = {"m": 10} if solver == "gmres" else {}
    x, info = getattr(oracle, solver)(rp, col, val, b, tol=1e-12, precond="block_jacobi", block_size=bs, **kw)
    assert info.status == oracle.CONVERGED and info.iterations == 1, info
    assert np.allclose(x, np.linalg.solve(a, b), rtol=0, atol=1e-11 * np.abs(np.linalg.solve(a, b)).max())


def _random_block_diag(rng, n, bs):
    blocks = []
    for _ in range(0, n, bs):
        g = rng.standard_normal((bs, bs))
        blocks.append(g + 3 * bs * np.eye(bs))
    return _block_diag(np.array(blocks), n)


@pytest.mark.parametrize("solver", ["bicgstab", "cgs", "gmres"])
@pytest.mark.parametrize("j", [3, 7])
def test_right_block_jacobi_invariant_under_block_column_scaling(solver, j):
    bs = 4
    rp, col, val = synth.convdiff3d_upwind(5)
    a = to_dense(rp, col, val)
    n = a.shape[0]
    rng = np.random.default_rng(21 + j)
    s = _random_block_diag(rng, n, bs)
    b = rng.standard_normal(n)
    rps, cols, vals = csr_from_dense(a @ s)
    kw = {"m": 40} if solver == "gmres" else {}
    x, _ = getattr(oracle, solver)(rp, col, val, b, tol=0.0, maxit=j, precond="block_jacobi", block_size=bs, **kw)
    xs, _ = getattr(oracle, solver)(rps, cols, vals, b, tol=0.0, maxit=j, precond="block_jacobi", block_size=bs,
                                    **kw)
    assert np.linalg.norm(s @ xs - x) <= 1e-9 * np.linalg.norm(x)
    # without the preconditioner the scaling changes the iterates
    xu, _ = getattr(oracle, solver)(rp, col, val, b, tol=0.0, maxit=j, **kw)
    xus, _ = getattr(oracle, solver)(rps, cols, vals, b, tol=0.0, maxit=j, **kw)
    assert np.linalg.norm(s @ xus - xu) > 1e-3 * np.linalg.norm(xu)


@pytest.mark.parametrize("j", [2, 5, 9])
def test_block_pcg_invariant_under_symmetric_block_scaling(j):
    bs = 4
    rp, col, val = synth.laplace2d_5pt(8)
    a = to_dense(rp, col, val)
    n = a.shape[0]
    rng = np.random.default_rng(40 + j)
    s = _random_block_diag(rng, n, bs)
    b = rng.standard_normal(n)
    rps, cols, vals = csr_from_dense(s.T @ a @ s)
    x, _ = oracle.cg(rp, col, val, b, tol=0.0, maxit=j, precond="block_jacobi", block_size=bs)
    xs, _ = oracle.cg(rps, cols, vals, s.T @ b, tol=0.0, maxit=j, precond="block_jacobi", block_size=bs)
    assert np.linalg.norm(s @ xs - x) <= 1e-9 * np.linalg.norm(x)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "gmres"])
def test_block_jacobi_beats_jacobi_on_block_coupled_matrix(solver):
    """A matrix whose strong couplings sit inside the blocks: block-Jacobi
    removes them, Jacobi cannot, so it needs fewer iterations."""
    bs = 8
    rp, col, val = synth.laplace2d_5pt(24)
    a = to_dense(rp, col, val)
    n = a.shape[0]
    rng = np.random.default_rng(77)
    inner = _random_block_diag(rng, n, bs)
    inner = inner @ inner.T if solver == "cg" else inner
    a = a + 20 * inner
    rp2, col2, val2 = csr_from_dense(a)
    b = rng.standard_normal(n)
    kw = {"m": 30} if solver == "gmres" else {}
    _, ij = getattr(oracle, solver)(rp2, col2, val2, b, tol=1e-10, maxit=5000, precond="jacobi", **kw)
    xb, ib = getattr(oracle, solver)(rp2, col2, val2, b, tol=1e-10, maxit=5000, precond="block_jacobi",
                                     block_size=bs, **kw)
    assert ib.status == oracle.CONVERGED and ib.iterations < ij.iterations, (ib, ij)
    assert np.linalg.norm(b - a @ xb) <= 1e-10 * np.linalg.norm(b)


def test_planted_transposed_block_is_caught():
    """The oracle rebuilt with the blocks applied transposed (mutant 8) fails
    the one-step pin on nonsymmetric blocks that the correct oracle passes."""
    bs = 4
    rng = np.random.default_rng(8)
    n = 4 * bs
    a = np.zeros((n, n))
    for c0 in range(0, n, bs):
        a[c0:c0 + bs, c0:c0 + bs] = rng.standard_normal((bs, bs)) + 2 * bs * np.eye(bs)
    rp, col, val = csr_from_dense(a)
    b = rng.standard_normal(n)
    _, good = oracle.bicgstab(rp, col, val, b, tol=1e-12, precond="block_jacobi", block_size=bs)
    _, bad = oracle.bicgstab(rp, col, val, b, tol=1e-12, precond="block_jacobi", block_size=bs, mutant=8)
    assert good.iterations == 1 and bad.iterations > 1


# ---------------------------------------------------------------- adaptive storage
# Reading (the paper cites adaptive-precision block-Jacobi without a rule): a
# block's inverse is stored in FP32 when kappa_1(D_k) * 2^-24 <= 1e-2, else FP64.

def test_adaptive_flags_follow_the_condition_number():
    # block k = diag(1, ..., 1, c_k): kappa_1 = c_k exactly
    bs = 4
    cs = [1.0, 1e3, 1.6e5, 1.7e5, 1e8, 3.0]
    d = np.ones(bs * len(cs))
    for k, c in enumerate(cs):
        d[k * bs + bs - 1] = c
    a = np.diag(d)
    rp, col, val = csr_from_dense(a)
    inv, flags = oracle.block_jacobi_inv(rp, col, val, bs, adaptive=True)
    want = [int(c * 2.0**-24 > 1e-2) for c in cs]
    assert flags.tolist() == want == [0, 0, 0, 1, 1, 0]
    for k, c in enumerate(cs):
        e = inv[k][bs - 1, bs - 1]
        assert e == (1.0 / c if want[k] else float(np.float32(1.0 / c)))


def test_adaptive_fp32_blocks_stay_within_the_bound():
    rng = np.random.default_rng(12)
    bs, n = 8, 8 * 40
    a = np.zeros((n, n))
    for k, c0 in enumerate(range(0, n, bs)):
        g = rng.standard_normal((bs, bs))
        if k % 3 == 0:  # every third block ill-conditioned: kappa ~ 1e7
            q, _ = np.linalg.qr(g)
            a[c0:c0 + bs, c0:c0 + bs] = q @ np.diag(np.geomspace(1.0, 1e-7, bs)) @ q.T
        else:
            a[c0:c0 + bs, c0:c0 + bs] = g + rng.choice([3.0, 30.0]) * np.eye(bs)
    rp, col, val = csr_from_dense(a)
    inv, flags = oracle.block_jacobi_inv(rp, col, val, bs, adaptive=True)
    exact = oracle.block_jacobi_inv(rp, col, val, bs)
    assert flags.tolist() == [int(k % 3 == 0) for k in range(n // bs)]
    for k in range(n // bs):
        blk = a[k * bs:(k + 1) * bs, k * bs:(k + 1) * bs]
        kappa = np.linalg.norm(blk, 1) * np.linalg.norm(np.linalg.inv(blk), 1)
        assert flags[k] == int(kappa * 2.0**-24 > 1e-2)
        if flags[k]:
            assert np.array_equal(inv[k], exact[k])
        else:
            assert np.array_equal(inv[k], exact[k].astype(np.float32).astype(np.float64))
            assert np.linalg.norm(blk @ inv[k] - np.eye(bs), 1) <= 1e-2


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_adaptive_all_fp64_blocks_equals_block_jacobi(solver):
    # blocks with kappa > 1.7e5: every one stays FP64, the solve is the FP64 one bit for bit
    bs = 4
    rng = np.random.default_rng(3)
    n = 4 * 30
    a = np.zeros((n, n))
    for c0 in range(0, n, bs):
        q, _ = np.linalg.qr(rng.standard_normal((bs, bs)))
        s = np.diag([1.0, 10.0, 1e3, 1e6])
        blk = q @ s @ q.T
        a[c0:c0 + bs, c0:c0 + bs] = blk if solver == "cg" else blk + 0.1 * rng.standard_normal((bs, bs))
    a += np.diag(np.full(n - 1, 0.01), 1) + np.diag(np.full(n - 1, 0.01), -1)
    rp, col, val = csr_from_dense(a)
    _, flags = oracle.block_jacobi_inv(rp, col, val, bs, adaptive=True)
    assert flags.all()
    b = rng.standard_normal(n)
    kw = {"m": 20} if solver == "gmres" else {}
    x1, i1 = getattr(oracle, solver)(rp, col, val, b, tol=0.0, maxit=6, precond="block_jacobi", block_size=bs, **kw)
    x2, i2 = getattr(oracle, solver)(rp, col, val, b, tol=0.0, maxit=6, precond="adaptive_block_jacobi",
                                     block_size=bs, **kw)
    assert np.array_equal(x1, x2)


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_adaptive_block_diagonal_converges_in_few_steps(solver):
    # well-conditioned blocks go to FP32: M^-1 A = I + O(1e-7), so each step
    # gains about seven digits instead of converging in one
    bs = 8
    rng = np.random.default_rng(5)
    n = bs * 30 + 5
    a = np.zeros((n, n))
    for c0 in range(0, n, bs):
        k = min(bs, n - c0)
        a[c0:c0 + k, c0:c0 + k] = rng.standard_normal((k, k)) + 2 * k * np.eye(k)
    rp, col, val = csr_from_dense(a)
    _, flags = oracle.block_jacobi_inv(rp, col, val, bs, adaptive=True)
    assert not flags.any()
    b = rng.standard_normal(n)
    kw = {"m": 10} if solver == "gmres" else {}
    x, info = getattr(oracle, solver)(rp, col, val, b, tol=1e-12, precond="adaptive_block_jacobi", block_size=bs,
                                      **kw)
    # (a BiCGSTAB iteration applies the preconditioner twice)
    lo, hi = (2, 3) if solver == "gmres" else (1, 2)
    assert info.status == oracle.CONVERGED and lo <= info.iterations <= hi, info
    assert np.allclose(x, np.linalg.solve(a, b), rtol=0, atol=1e-11)


def test_adaptive_needs_fp32_range():
    # kappa = 1, but the inverse of 1e-40 * I overflows FP32 (and that of 1e39 * I
    # is subnormal in FP32): both stay FP64; a moderate scale goes to FP32
    bs = 2
    d = np.array([1e-40, 1e-40, 1e39, 1e39, 3.0, 3.0])
    rp, col, val = csr_from_dense(np.diag(d))
    inv, flags = oracle.block_jacobi_inv(rp, col, val, bs, adaptive=True)
    assert flags.tolist() == [1, 1, 0]
    assert inv[0][0, 0] == 1e40 and inv[1][0, 0] == 1.0 / 1e39
