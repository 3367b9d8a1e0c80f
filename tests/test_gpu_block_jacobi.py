"""GPU block-Jacobi preconditioning against the CPU oracle.

Element-by-element parity of the iterates after a few fixed iterations (the
block inverses, their application and each solver's use of them), one-step
convergence on block-diagonal matrices, solves to 1e-10 with the oracle's
iteration counts on every storage format, block sizes 1 to 32 with a ragged
last block, singular blocks, refinement and FP32, and invalid block sizes."""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import to_dense, residual_limit

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


def _make(spx, ctx, fmt, rp, col, val, flags=0, dtype=None):
    v = _t(val) if dtype is None else _t(val).to(dtype)
    return spx.spx_matrix_create(ctx, fmt, _t(rp), _t(col), v, flags=flags)


def csr_from_dense(a):
    r, c = np.nonzero(a)
    rp = np.zeros(a.shape[0] + 1, dtype=np.int32)
    np.cumsum(np.bincount(r, minlength=a.shape[0]), out=rp[1:])
    return rp, c.astype(np.int32), a[r, c].astype(np.float64)


def _relres(rp, col, val, b, x):
    return np.linalg.norm(b - oracle.spmv_csr(rp, col, val, x)) / np.linalg.norm(b)


def _coupled(solver, m=11, bs=8, seed=31):
    """Upwind convection-diffusion (m^3 rows, ragged for every bs > 1) plus strong
    couplings inside the diagonal blocks of size bs (random, scaled and shifted
    so that every block stays well conditioned: the iterates then move by
    ~1e-14 under a 1e-15 perturbation of A); a 3D Laplacian plus random
    positive semidefinite blocks for CG."""
    rng = np.random.default_rng(seed)
    if solver == "cg":
        rp, col, val = synth.laplace3d_7pt(m)
    else:
        rp, col, val = synth.convdiff3d_upwind(m, peclet=10.0)
    a = to_dense(rp, col, val)
    n = a.shape[0]
    blocks = np.zeros((n, n))
    for c0 in range(0, n, bs):
        k = min(bs, n - c0)
        g = rng.standard_normal((k, k)) / np.sqrt(k)  # eigenvalues near the unit disc
        blocks[c0:c0 + k, c0:c0 + k] = 2.25 * (g @ g.T) if solver == "cg" else 1.5 * g + 2.0 * np.eye(k)
    a = a + 4.0 * blocks
    rp, col, val = csr_from_dense(a)
    xs = synth.uniform_vector(n, seed=3)
    return rp, col, val, xs, oracle.spmv_csr(rp, col, val, xs)


def _oracle(solver, rp, col, val, b, **kw):
    if solver == "gmres":
        return oracle.gmres(rp, col, val, b, m=30, **kw)
    return getattr(oracle, solver)(rp, col, val, b, **kw)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
@pytest.mark.parametrize("bs", [1, 2, 4, 8, 16, 32])
def test_fixed_iterations_match_oracle_elementwise(spx, ctx, solver, bs):
    rp, col, val, xs, b = _coupled(solver, m=9, bs=bs)
    n = b.shape[0]
    j = 4
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        spx.spx_solve_fixed(ctx, A, _t(b), x, solver, j, restart=30, precond="block_jacobi", block_size=bs)
        xo, _ = _oracle(solver, rp, col, val, b, tol=0.0, maxit=j, precond="block_jacobi", block_size=bs)
        xg = x.cpu().numpy()
        assert np.allclose(xg, xo, rtol=0, atol=1e-9 * np.abs(xo).max()), np.abs(xg - xo).max()
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
@pytest.mark.parametrize("bs", [4, 32])
def test_block_diagonal_matrix_one_step(spx, ctx, solver, bs):
    rng = np.random.default_rng(bs + 1)
    n = 40 * bs + 3  # ragged last block
    a = np.zeros((n, n))
    for c0 in range(0, n, bs):
        k = min(bs, n - c0)
        g = rng.standard_normal((k, k))
        a[c0:c0 + k, c0:c0 + k] = g @ g.T + k * np.eye(k) if solver == "cg" else g + 2 * k * np.eye(k)
    rp, col, val = csr_from_dense(a)
    b = rng.standard_normal(n)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-12, 100, restart=10, precond="block_jacobi",
                             block_size=bs)
        assert info.status == spx.SPX_CONVERGED and info.iterations == 1, info
        want = np.linalg.solve(a, b)
        assert np.allclose(x.cpu().numpy(), want, rtol=0, atol=1e-11 * np.abs(want).max())
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo", "hyb"])
@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_block_jacobi_solve_matches_oracle(spx, ctx, solver, fmt):
    bs = 8
    rp, col, val, xs, b = _coupled(solver, bs=bs)
    A = _make(spx, ctx, fmt, rp, col, val)
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 20000, restart=30, precond="block_jacobi",
                             block_size=bs)
        _, oinfo = _oracle(solver, rp, col, val, b, tol=1e-10, maxit=20000, precond="block_jacobi", block_size=bs)
        assert info.status == spx.SPX_CONVERGED and oinfo.status == oracle.CONVERGED, (info, oinfo)
        assert info.relres_true <= 1e-10 and _relres(rp, col, val, b, x.cpu().numpy()) <= residual_limit(rp, col, val, b, x.cpu().numpy(), 1e-10)
        slack = max(4, oinfo.iterations // (5 if solver == "cgs" else 10))
        assert abs(info.iterations - oinfo.iterations) <= slack, (info, oinfo)
        # the blocks carry the strong couplings: block-Jacobi beats Jacobi
        _, jinfo = _oracle(solver, rp, col, val, b, tol=1e-10, maxit=20000, precond="jacobi")
        assert jinfo.status != oracle.CONVERGED or jinfo.iterations > info.iterations
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_bs1_block_jacobi_follows_jacobi(spx, ctx, solver):
    rp, col, val, xs, b = _coupled(solver, bs=4)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        out = []
        for kw in ({"precond": "jacobi"}, {"precond": "block_jacobi", "block_size": 1}):
            x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
            info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 20000, restart=30, **kw)
            assert info.status == spx.SPX_CONVERGED
            out.append((info, x.cpu().numpy()))
        assert abs(out[0][0].iterations - out[1][0].iterations) <= 2
        assert np.allclose(out[0][1], out[1][1], rtol=0, atol=1e-6 * np.abs(out[0][1]).max())
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["bicgstab", "cgs", "gmres"])
def test_right_block_jacobi_block_scaling_invariance_on_gpu(spx, ctx, solver):
    bs = 4
    rp, col, val = synth.convdiff3d_upwind(7, peclet=10.0)
    a = to_dense(rp, col, val)
    n = a.shape[0]
    rng = np.random.default_rng(17)
    s = np.zeros((n, n))
    for c0 in range(0, n, bs):
        k = min(bs, n - c0)
        s[c0:c0 + k, c0:c0 + k] = rng.standard_normal((k, k)) + 3 * k * np.eye(k)
    b = rng.standard_normal(n)
    xs = []
    for mat in (a, a @ s):
        rpc, colc, valc = csr_from_dense(mat)
        A = _make(spx, ctx, "csr", rpc, colc, valc)
        try:
            x = torch.zeros(n, dtype=torch.float64, device=DEV)
            spx.spx_solve_fixed(ctx, A, _t(b), x, solver, 6, restart=30, precond="block_jacobi", block_size=bs)
            xs.append(x.cpu().numpy())
        finally:
            spx.spx_matrix_destroy(A)
    assert np.linalg.norm(s @ xs[1] - xs[0]) <= 1e-8 * np.linalg.norm(xs[0])


def test_singular_block_counts_as_identity(spx, ctx):
    n = 64
    rng = np.random.default_rng(6)
    a = np.diag(rng.uniform(2.0, 4.0, n))
    a[8:16, 8:16] = 0.0
    a[8:16, 8] = rng.uniform(1.0, 2.0, 8)  # block 1: one nonzero column, exactly singular
    for i in range(8, 16):  # couple blocks 1 and 2 so that A itself is well conditioned
        a[i, i + 8] += 5.0
        a[i + 8, i] += 5.0
    assert np.linalg.cond(a) < 1e2
    rp, col, val = csr_from_dense(a)
    assert np.array_equal(oracle.block_jacobi_inv(rp, col, val, 8)[1], np.eye(8))
    b = rng.standard_normal(n)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        spx.spx_solve_fixed(ctx, A, _t(b), x, "gmres", 5, restart=10, precond="block_jacobi", block_size=8)
        xo, _ = oracle.gmres(rp, col, val, b, m=10, tol=0.0, maxit=5, precond="block_jacobi", block_size=8)
        assert np.allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-10 * np.abs(xo).max())
        x.zero_()
        info = spx.spx_solve(ctx, A, _t(b), x, "gmres", 1e-12, 200, restart=30, precond="block_jacobi",
                             block_size=8)
        assert info.status == spx.SPX_CONVERGED
        assert np.allclose(x.cpu().numpy(), np.linalg.solve(a, b), rtol=0, atol=1e-11)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_block_jacobi_mixed_precision(spx, ctx, solver):
    rp, col, val, xs, b = _coupled(solver, bs=8)
    A = _make(spx, ctx, "csr", rp, col, val, flags=spx.SPX_MIXED_SHADOW)
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 20000, restart=30, precision="mixed",
                             precond="block_jacobi", block_size=8)
        assert info.status == spx.SPX_CONVERGED, info
        assert _relres(rp, col, val, b, x.cpu().numpy()) <= residual_limit(rp, col, val, b, x.cpu().numpy(), 1e-10)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "gmres"])
def test_block_jacobi_fp32(spx, ctx, solver):
    rp, col, val, xs, b = _coupled(solver, bs=16)
    A = _make(spx, ctx, "csr", rp, col, val, dtype=torch.float32)
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float32, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b).float(), x, solver, 1e-5, 5000, restart=30, precision="f32",
                             precond="block_jacobi", block_size=16)
        assert info.status == spx.SPX_CONVERGED, info
        v32 = val.astype(np.float32).astype(np.float64)
        b32 = b.astype(np.float32).astype(np.float64)
        assert _relres(rp, col, v32, b32, x.double().cpu().numpy()) <= 2e-5
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("bs", [0, 3, 64])
def test_invalid_block_size_is_rejected(spx, ctx, bs):
    rp, col, val, xs, b = _coupled("cg", m=5, bs=4)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        with pytest.raises(spx.SpxError) as ei:
            spx.spx_solve(ctx, A, _t(b), x, "cg", 1e-10, 100, precond="block_jacobi", block_size=bs)
        assert ei.value.status == spx.SPX_ERR_INVALID
    finally:
        spx.spx_matrix_destroy(A)


# ---------------------------------------------------------------- adaptive storage
def _alternating(solver, bs, nblk=60, seed=7):
    """Block-diagonal A whose even blocks (kappa ~ 3e3) are stored in FP32 and
    odd ones (kappa ~ 1e6) in FP64; b takes each FP32 block's leading left
    singular vector, where rounding the inverse to FP32 shows most (~kappa *
    2^-24), and random entries elsewhere."""
    rng = np.random.default_rng(seed)
    n = bs * nblk + bs // 2
    a = np.zeros((n, n))
    b = np.zeros(n)
    for k, c0 in enumerate(range(0, n, bs)):
        kk = min(bs, n - c0)
        q1, _ = np.linalg.qr(rng.standard_normal((kk, kk)))
        q2 = q1 if solver == "cg" else np.linalg.qr(rng.standard_normal((kk, kk)))[0]
        fp64 = bool(k % 2) and kk > 1
        sv = np.geomspace(1.0, 1e-6 if fp64 else 3e-4, kk) if kk > 1 else np.ones(1)
        a[c0:c0 + kk, c0:c0 + kk] = q1 @ np.diag(sv) @ q2.T
        b[c0:c0 + kk] = rng.standard_normal(kk) if fp64 else q1[:, 0]
    return a, b


def _block_rel(x, y, bs):
    return np.array([np.linalg.norm(x[c:c + bs] - y[c:c + bs]) / np.linalg.norm(y[c:c + bs])
                     for c in range(0, len(y), bs)])


@pytest.mark.parametrize("solver", ["cg", "gmres"])
@pytest.mark.parametrize("bs", [2, 4, 8, 32])
def test_adaptive_storage_reads_each_block_from_its_precision(spx, ctx, solver, bs):
    a, b = _alternating(solver, bs)
    rp, col, val = csr_from_dense(a)
    n = b.shape[0]
    _, flags = oracle.block_jacobi_inv(rp, col, val, bs, adaptive=True)
    assert flags.tolist() == [int(k % 2 == 1 and min(bs, n - k * bs) > 1) for k in range(len(flags))]
    kw = {"m": 5} if solver == "gmres" else {}
    xo, _ = _oracle_1(solver, rp, col, val, b, "adaptive_block_jacobi", bs, kw)
    x64, _ = _oracle_1(solver, rp, col, val, b, "block_jacobi", bs, kw)
    # the FP32 blocks' rounding is visible at this right-hand side
    f32 = [k for k in range(len(flags)) if not flags[k] and min(bs, n - k * bs) > 1]
    assert _block_rel(x64, xo, bs)[f32].min() > 5e-8
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        spx.spx_solve_fixed(ctx, A, _t(b), x, solver, 1, restart=5, precond="adaptive_block_jacobi", block_size=bs)
        assert _block_rel(x.cpu().numpy(), xo, bs).max() <= 2e-8
    finally:
        spx.spx_matrix_destroy(A)


def _oracle_1(solver, rp, col, val, b, precond, bs, kw, j=1):
    return getattr(oracle, solver)(rp, col, val, b, tol=0.0, maxit=j, precond=precond, block_size=bs, **kw)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_adaptive_storage_fixed_iterations_match_oracle(spx, ctx, solver):
    bs = 8
    a, b = _alternating(solver, bs, seed=9)
    rp, col, val = csr_from_dense(a)
    kw = {"m": 5} if solver == "gmres" else {}
    xo, _ = _oracle_1(solver, rp, col, val, b, "adaptive_block_jacobi", bs, kw, j=3)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        spx.spx_solve_fixed(ctx, A, _t(b), x, solver, 3, restart=5, precond="adaptive_block_jacobi", block_size=bs)
        assert _block_rel(x.cpu().numpy(), xo, bs).max() <= 1e-6
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "cgs", "gmres"])
def test_adaptive_solve_matches_oracle(spx, ctx, solver):
    bs = 8
    rp, col, val, xs, b = _coupled(solver, bs=bs)
    _, flags = oracle.block_jacobi_inv(rp, col, val, bs, adaptive=True)
    assert not flags.any()  # well-conditioned blocks: all stored in FP32
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        x = torch.zeros(b.shape[0], dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-10, 20000, restart=30, precond="adaptive_block_jacobi",
                             block_size=bs)
        _, oinfo = _oracle(solver, rp, col, val, b, tol=1e-10, maxit=20000, precond="adaptive_block_jacobi",
                           block_size=bs)
        assert info.status == spx.SPX_CONVERGED and oinfo.status == oracle.CONVERGED, (info, oinfo)
        assert _relres(rp, col, val, b, x.cpu().numpy()) <= residual_limit(rp, col, val, b, x.cpu().numpy(), 1e-10)
        assert abs(info.iterations - oinfo.iterations) <= max(4, oinfo.iterations // 10), (info, oinfo)
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("solver", ["cg", "gmres"])
def test_adaptive_with_every_block_fp64_is_block_jacobi_bitwise(spx, ctx, solver):
    bs = 4
    rng = np.random.default_rng(3)
    n = bs * 50
    a = np.zeros((n, n))
    for c0 in range(0, n, bs):
        q, _ = np.linalg.qr(rng.standard_normal((bs, bs)))
        a[c0:c0 + bs, c0:c0 + bs] = q @ np.diag([1.0, 10.0, 1e3, 1e6]) @ q.T
    a += np.diag(np.full(n - 1, 0.01), 1) + np.diag(np.full(n - 1, 0.01), -1)
    rp, col, val = csr_from_dense(a)
    assert oracle.block_jacobi_inv(rp, col, val, bs, adaptive=True)[1].all()
    b = rng.standard_normal(n)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        out = []
        for pc in ("block_jacobi", "adaptive_block_jacobi"):
            x = torch.zeros(n, dtype=torch.float64, device=DEV)
            spx.spx_solve_fixed(ctx, A, _t(b), x, solver, 6, restart=20, precond=pc, block_size=bs)
            out.append(x.cpu().numpy())
        assert np.array_equal(out[0], out[1])
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("bs", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_block_inverse_with_row_pivoting_one_step(spx, ctx, solver, bs):
    """Blocks that are row permutations of diagonally dominant ones: their
    diagonals hold small or zero entries, so the inversion has to pivot."""
    rng = np.random.default_rng(50 + bs)
    n = 30 * bs + 1
    a = np.zeros((n, n))
    for c0 in range(0, n, bs):
        k = min(bs, n - c0)
        blk = 0.3 * rng.standard_normal((k, k)) + 3.0 * np.eye(k)
        perm = np.roll(np.arange(k), 1)  # a cyclic shift: every diagonal entry moves off the diagonal
        a[c0:c0 + k, c0:c0 + k] = blk[perm]
    rp, col, val = csr_from_dense(a)
    b = rng.standard_normal(n)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        for pc in ("block_jacobi", "adaptive_block_jacobi"):
            x = torch.zeros(n, dtype=torch.float64, device=DEV)
            info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-12, 100, restart=10, precond=pc, block_size=bs)
            assert info.status == spx.SPX_CONVERGED and info.iterations <= (1 if pc == "block_jacobi" else 3), info
            want = np.linalg.solve(a, b)
            assert np.allclose(x.cpu().numpy(), want, rtol=0, atol=1e-11 * np.abs(want).max())
    finally:
        spx.spx_matrix_destroy(A)


@pytest.mark.parametrize("n,bs", [(1, 1), (1, 8), (3, 32), (31, 16), (33, 32), (5, 4)])
@pytest.mark.parametrize("precond", ["block_jacobi", "adaptive_block_jacobi"])
def test_tiny_systems(spx, ctx, n, bs, precond):
    """Fewer rows than one block, one row, and ragged tails inside a single warp."""
    rng = np.random.default_rng(n * 100 + bs)
    a = rng.standard_normal((n, n)) + 2 * n * np.eye(n)
    rp, col, val = csr_from_dense(a)
    b = rng.standard_normal(n)
    A = _make(spx, ctx, "csr", rp, col, val)
    try:
        for solver in ("bicgstab", "gmres"):
            x = torch.zeros(n, dtype=torch.float64, device=DEV)
            info = spx.spx_solve(ctx, A, _t(b), x, solver, 1e-12, 100, restart=10, precond=precond, block_size=bs)
            assert info.status == spx.SPX_CONVERGED, (solver, info)
            want = np.linalg.solve(a, b)
            assert np.allclose(x.cpu().numpy(), want, rtol=0, atol=1e-11 * np.abs(want).max())
    finally:
        spx.spx_matrix_destroy(A)


def test_empty_system_with_block_jacobi(spx, ctx):
    rp = np.zeros(1, dtype=np.int32)
    A = spx.spx_matrix_create(ctx, "csr", _t(rp), torch.zeros(0, dtype=torch.int32, device=DEV),
                              torch.zeros(0, dtype=torch.float64, device=DEV))
    try:
        x = torch.zeros(0, dtype=torch.float64, device=DEV)
        info = spx.spx_solve(ctx, A, torch.zeros(0, dtype=torch.float64, device=DEV), x, "cg", 1e-10, 10,
                             precond="block_jacobi", block_size=8)
        assert info.status == spx.SPX_CONVERGED and info.iterations == 0
    finally:
        spx.spx_matrix_destroy(A)
